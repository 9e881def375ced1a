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
