"""IQ-DAS and BB-DMAS (Sec. II-B-1, Eq. (4)) on the GPU against the FP64 oracle.

The oracle demodulates the int16 records in float64; the library demodulates
them on the GPU in FP32 (length-Ns transforms), interpolates the analytic
signal and restores the carrier phase.  Magnitude images, so the bound is the
FP32 one: relative L2 1e-5 and 2e-5 of the peak per pixel.
"""
import numpy as np
import pytest

import oracle
import paper_2311_00482_gb300 as bf
import synth
from test_gpu_parity import assert_close, grid_of, make_handle, run_gpu

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


def iq_ref(acq, rf):
    iq = oracle.demodulate(rf, acq.fs_hz, acq.f0_hz)
    return oracle.beamform_iq(iq, acq.x_elements(), acq.angles_rad, grid_of(acq), acq.fs_hz,
                              acq.c_mps, acq.f_number, acq.f0_hz)


@pytest.mark.parametrize("rows", ["4", "8"])
def test_ragged_grid_both_iq_combiners(torch, monkeypatch, rows):
    monkeypatch.setenv("BF_TILE_ROWS", rows)
    acq = synth.SPECKLE_POINTS_128.with_(nx=100, nz=77, angles_deg=(-6.0, 0.0, 6.0))
    rf, _ = synth.speckle_points_frame(acq)
    ref = iq_ref(acq, rf)
    got = run_gpu(torch, acq, rf, bf.BF_IQDAS | bf.BF_BBDMAS)
    assert got.shape[0] == 2
    assert_close(got[0], ref["iqdas"], bf.BF_PREC_FP32, "iq-das rows=" + rows)
    assert_close(got[1], ref["bbdmas"], bf.BF_PREC_FP32, "bb-dmas rows=" + rows)


def test_full_size_512_iq_and_log(torch):
    acq = synth.CYST_WIRES_512
    rf, _ = synth.cyst_wires_frame(acq)
    ref = iq_ref(acq, rf)
    h = make_handle(acq)
    try:
        got = run_gpu(torch, acq, rf, bf.BF_IQDAS | bf.BF_BBDMAS, h=h)
        assert_close(got[0], ref["iqdas"], bf.BF_PREC_FP32, "iq-das")
        assert_close(got[1], ref["bbdmas"], bf.BF_PREC_FP32, "bb-dmas")
        env = run_gpu(torch, acq, rf, bf.BF_IQDAS | bf.BF_BBDMAS | bf.BF_OUT_ENV, h=h)
        np.testing.assert_array_equal(env, got)
        db = run_gpu(torch, acq, rf, bf.BF_IQDAS | bf.BF_BBDMAS | bf.BF_OUT_LOGDB, h=h)
        for k, name in enumerate(("iqdas", "bbdmas")):
            assert np.max(np.abs(db[k] - oracle.log_compress(ref[name]))) <= 0.05, name
    finally:
        bf.bf_destroy(h)


def test_single_combiners_and_subset_order(torch):
    acq = synth.SPECKLE_POINTS_128.with_(nx=40, nz=90, angles_deg=(4.0,))
    rf, _ = synth.speckle_points_frame(acq)
    ref = iq_ref(acq, rf)
    got = run_gpu(torch, acq, rf, bf.BF_BBDMAS)
    assert got.shape[0] == 1
    assert_close(got[0], ref["bbdmas"], bf.BF_PREC_FP32, "bb-dmas alone")
    got = run_gpu(torch, acq, rf, bf.BF_IQDAS)
    assert_close(got[0], ref["iqdas"], bf.BF_PREC_FP32, "iq-das alone")


def test_iq_in_a_batch_equals_single_frames(torch):
    acqs = [synth.SPECKLE_POINTS_128.with_(nx=48, nz=64),
            synth.CYST_WIRES_512.with_(nx=96, nz=128, angles_deg=(-5.0, 5.0))]
    frames, handles, keep, singles = [], [], [], []
    try:
        for k, acq in enumerate(acqs):
            rf = (synth.speckle_points_frame(acq)[0] if k == 0 else synth.cyst_wires_frame(acq)[0])
            h = make_handle(acq)
            handles.append(h)
            flags = bf.BF_IQDAS | bf.BF_BBDMAS | bf.BF_OUT_LOGDB
            rf_d = torch.from_numpy(rf).cuda()
            out = torch.zeros((2, acq.nx, acq.nz), device="cuda")
            keep += [rf_d, out]
            frames.append((h, rf_d, acq.n_samples, acq.angles_rad, flags, out))
            singles.append(run_gpu(torch, acq, rf, flags, h=h))
        batch = bf.Batch(frames)
        batch.launch()
        batch.status()
        for (h, rf_d, ns, ang, flags, out), ref in zip(frames, singles):
            np.testing.assert_array_equal(out.cpu().numpy(), ref.astype(np.float32))
        batch.close()
    finally:
        for h in handles:
            bf.bf_destroy(h)


def test_iq_argument_checks(torch):
    acq = synth.SPECKLE_POINTS_128.with_(nx=16, nz=16)
    h = make_handle(acq)
    try:
        rf = torch.zeros((1, 64, 1024), dtype=torch.int16, device="cuda")
        out = torch.zeros((2, 16, 16), device="cuda")
        bad = [bf.BF_IQDAS | bf.BF_DAS, bf.BF_IQDAS | bf.BF_PREC_FP16]
        for flags in bad:
            with pytest.raises(bf.BFError):
                bf.bf_beamform(h, rf, 1024, [0.0], flags, out)
        rf3 = torch.zeros((1, 64, 1000), dtype=torch.int16, device="cuda")
        with pytest.raises(bf.BFError):
            bf.bf_beamform(h, rf3, 1000, [0.0], bf.BF_IQDAS, out)
        with pytest.raises(bf.BFError):
            bf.bf_beamform_plain(h, rf, 1024, [0.0], bf.BF_IQDAS, out)
    finally:
        bf.bf_destroy(h)


def assert_db_close(got, mag, what):
    """dB image against the oracle's magnitude image `mag`: per pixel within the
    first-order change of 20 log10(mag / max) under a magnitude error
    E = 2e-6 of the peak, 8.686 E / max(mag, 10^(-70/20) peak) + 8.686 E / peak
    (0.055 dB at the -70 dB floor)."""
    peak = float(mag.max())
    e = 2e-6 * peak
    tol = 8.686 * e / np.maximum(mag, 10 ** (-70 / 20) * peak) + 8.686 * e / peak
    err = np.abs(got - oracle.log_compress(mag))
    assert np.all(err <= tol), "%s: %d pixels off, worst %.3f dB" % (what, int((err > tol).sum()),
                                                                     float(err.max()))


def assert_matches_single(got, single, is_db, what):
    """A frame of a multi-frame job against the same frame beamformed alone.
    The beamforming arithmetic per frame is the single-frame kernel's, but a
    frame pair is demodulated in one complex transform (two real records),
    which rounds differently from one transform per record: magnitudes within
    2e-6 of the image's peak, dB images within 0.01 dB (a frame in the wrong
    place would be off by whole decibels)."""
    for m in range(got.shape[0]):
        atol = 0.01 if is_db else 2e-6 * float(np.max(np.abs(single[m])))
        np.testing.assert_allclose(got[m], single[m], rtol=0, atol=atol + 1e-30,
                                   err_msg="%s image %d" % (what, m))


def scaled_frames(acq, n, seed0):
    """n distinct records, frame k at (k + 2) / (n + 1) of its synthesized amplitude,
    so that the frames' image maxima (and dB images) differ."""
    out = []
    for k in range(n):
        rf = synth.speckle_points_frame(acq, seed=seed0 + k)[0].astype(np.float64)
        out.append(np.round(rf * (k + 2) / (n + 1)).astype(np.int16))
    return out


# (tile rows, frames, depth): seven frames on 16-row tiles make one four-frame
# job, one two-frame job and one frame alone; five on 32-row tiles two
# two-frame jobs and one alone.  Depth 92 with aligned images takes the
# bulk-copy epilogue, 90 the row-pair stores, 91 the per-pixel stores.
@pytest.mark.parametrize("rows,n,nz", [("2", 7, 92), ("2", 7, 90), ("2", 7, 91), ("4", 5, 92)])
def test_iq_frames_share_delay_and_carrier_phase(torch, monkeypatch, rows, n, nz):
    """Multi-frame IQ jobs (Sec. II-B-1, Eq. (4)): every frame's IQ-DAS and
    BB-DMAS images match the oracle and the frame's single-frame result on
    the same tiles, and the log stage normalises each frame by its own
    maximum."""
    monkeypatch.setenv("BF_TILE_ROWS", rows)
    acq = synth.SPECKLE_POINTS_128.with_(nx=70, nz=nz, angles_deg=(-4.0, 4.0))
    rfs = scaled_frames(acq, n, synth.BASE_SEED + 900)
    flags = bf.BF_IQDAS | bf.BF_BBDMAS
    h = make_handle(acq)
    try:
        assert bf.bf_plan_info(h, acq.n_samples, acq.angles_rad, flags)["rows"] == int(rows)
        rf_d = [torch.from_numpy(r).cuda() for r in rfs]
        for stage in (bf.BF_OUT_RF, bf.BF_OUT_LOGDB):
            outs = [torch.full((2, acq.nx, acq.nz), float("nan"), device="cuda") for _ in rfs]
            batch = bf.Batch([(h, rf_d[k], acq.n_samples, acq.angles_rad, flags | stage, outs[k])
                              for k in range(n)])
            try:
                batch.launch()
                batch.status()
                got = [o.cpu().numpy().astype(np.float64) for o in outs]
            finally:
                batch.close()
            for k in range(n):
                ref = iq_ref(acq, rfs[k])
                single = run_gpu(torch, acq, rfs[k], flags | stage, h=h)
                assert_matches_single(got[k], single, stage == bf.BF_OUT_LOGDB,
                                      "frame %d stage %d" % (k, stage))
                for m, name in enumerate(("iqdas", "bbdmas")):
                    if stage == bf.BF_OUT_RF:
                        assert_close(got[k][m], ref[name], bf.BF_PREC_FP32, "%s %d" % (name, k))
                    else:
                        assert_db_close(got[k][m], ref[name], "%s dB %d" % (name, k))
    finally:
        bf.bf_destroy(h)


@pytest.mark.parametrize("flags", [bf.BF_IQDAS, bf.BF_BBDMAS])
def test_iq_multi_frame_single_combiner(torch, monkeypatch, flags):
    """Four-frame jobs with one IQ combiner: every frame against the oracle."""
    monkeypatch.setenv("BF_TILE_ROWS", "2")
    acq = synth.SPECKLE_POINTS_128.with_(nx=40, nz=64, angles_deg=(3.0,))
    rfs = scaled_frames(acq, 4, synth.BASE_SEED + 920)
    name = "iqdas" if flags == bf.BF_IQDAS else "bbdmas"
    h = make_handle(acq)
    try:
        rf_d = [torch.from_numpy(r).cuda() for r in rfs]
        outs = [torch.full((1, acq.nx, acq.nz), float("nan"), device="cuda") for _ in rfs]
        batch = bf.Batch([(h, rf_d[k], acq.n_samples, acq.angles_rad, flags, outs[k])
                          for k in range(4)])
        try:
            batch.launch()
            batch.status()
        finally:
            batch.close()
        for k in range(4):
            assert_close(outs[k].cpu().numpy()[0].astype(np.float64), iq_ref(acq, rfs[k])[name],
                         bf.BF_PREC_FP32, "%s %d" % (name, k))
    finally:
        bf.bf_destroy(h)


def test_iq_job_with_mixed_output_stages(torch, monkeypatch):
    """Frames of one plan asking for different outputs share a job: the
    log-compressed frames get their own maxima, the magnitude frames none."""
    monkeypatch.setenv("BF_TILE_ROWS", "2")
    acq = synth.SPECKLE_POINTS_128.with_(nx=48, nz=80, angles_deg=(0.0,))
    rfs = scaled_frames(acq, 4, synth.BASE_SEED + 940)
    base = bf.BF_IQDAS | bf.BF_BBDMAS
    stages = [bf.BF_OUT_LOGDB, bf.BF_OUT_RF, bf.BF_OUT_LOGDB, bf.BF_OUT_ENV]
    h = make_handle(acq)
    try:
        rf_d = [torch.from_numpy(r).cuda() for r in rfs]
        outs = [torch.full((2, acq.nx, acq.nz), float("nan"), device="cuda") for _ in rfs]
        batch = bf.Batch([(h, rf_d[k], acq.n_samples, acq.angles_rad, base | stages[k], outs[k])
                          for k in range(4)])
        try:
            batch.launch()
            batch.status()
        finally:
            batch.close()
        for k in range(4):
            got = outs[k].cpu().numpy().astype(np.float64)
            assert_matches_single(got, run_gpu(torch, acq, rfs[k], base | stages[k], h=h),
                                  stages[k] == bf.BF_OUT_LOGDB, "frame %d" % k)
            ref = iq_ref(acq, rfs[k])
            for m, name in enumerate(("iqdas", "bbdmas")):
                if stages[k] == bf.BF_OUT_LOGDB:
                    assert_db_close(got[m], ref[name], "%s dB %d" % (name, k))
                else:
                    assert_close(got[m], ref[name], bf.BF_PREC_FP32, "%s %d" % (name, k))
    finally:
        bf.bf_destroy(h)


def test_iq_records_too_long_for_frame_pairs_run_alone(torch, monkeypatch):
    """8192-sample records: a frame pair's demodulation would need four 64 KB
    transform buffers in one CTA, so such IQ frames take one-frame jobs even
    on 16-row tiles; a batch of three still matches the oracle and equals the
    frames beamformed alone."""
    monkeypatch.setenv("BF_TILE_ROWS", "2")
    acq = synth.SPECKLE_POINTS_128.with_(nx=24, nz=40, n_samples=8192, z0_m=20e-3, z1_m=25e-3,
                                         angles_deg=(2.0,))
    rfs = scaled_frames(acq, 3, synth.BASE_SEED + 960)
    flags = bf.BF_IQDAS | bf.BF_BBDMAS
    h = make_handle(acq)
    try:
        assert bf.bf_plan_info(h, acq.n_samples, acq.angles_rad, flags)["rows"] == 2
        rf_d = [torch.from_numpy(r).cuda() for r in rfs]
        outs = [torch.full((2, acq.nx, acq.nz), float("nan"), device="cuda") for _ in rfs]
        batch = bf.Batch([(h, rf_d[k], acq.n_samples, acq.angles_rad, flags, outs[k])
                          for k in range(3)])
        try:
            batch.launch()
            batch.status()
        finally:
            batch.close()
        for k in range(3):
            got = outs[k].cpu().numpy().astype(np.float64)
            np.testing.assert_array_equal(got, run_gpu(torch, acq, rfs[k], flags, h=h))
            ref = iq_ref(acq, rfs[k])
            assert_close(got[0], ref["iqdas"], bf.BF_PREC_FP32, "iqdas %d" % k)
            assert_close(got[1], ref["bbdmas"], bf.BF_PREC_FP32, "bbdmas %d" % k)
    finally:
        bf.bf_destroy(h)
