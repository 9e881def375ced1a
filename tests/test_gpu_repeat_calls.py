"""Repeated bf_beamform calls: the handle keeps its last call and replays it
(after the first repetition as one CUDA graph).  A replay must read the
current contents of the buffers, and any change of plan, flags, buffers, order
p or stream must prepare the call afresh."""
import numpy as np
import pytest

import oracle
import paper_2311_00482_gb300 as bf
import synth
from test_gpu_parity import assert_close, make_handle, oracle_all

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


def test_repeats_follow_the_data_and_every_argument(torch):
    acq = synth.SPECKLE_POINTS_128.with_(nx=64, nz=96, angles_deg=(-5.0, 5.0))
    rf1, _ = synth.speckle_points_frame(acq)
    rf2, _ = synth.speckle_points_frame(acq, seed=synth.BASE_SEED + 77)
    ref1, ref2 = oracle_all(acq, rf1), oracle_all(acq, rf2)
    flags = bf.BF_DAS | bf.BF_DMAS
    h = make_handle(acq)
    try:
        rf_d = torch.from_numpy(rf1).cuda()
        out = torch.zeros((2, acq.nx, acq.nz), device="cuda")
        for _ in range(4):  # eager, then replay, then graph replays
            out.zero_()
            bf.bf_beamform(h, rf_d, acq.n_samples, acq.angles_rad, flags, out)
            bf.bf_sync(h)
            got = out.cpu().numpy().astype(np.float64)
            assert_close(got[0], ref1["das"], bf.BF_PREC_FP32, "das")
            assert_close(got[1], ref1["dmas"], bf.BF_PREC_FP32, "dmas")
        # new data in the same buffer: the replay reads it
        rf_d.copy_(torch.from_numpy(rf2))
        bf.bf_beamform(h, rf_d, acq.n_samples, acq.angles_rad, flags, out)
        bf.bf_sync(h)
        assert_close(out.cpu().numpy()[0].astype(np.float64), ref2["das"], bf.BF_PREC_FP32, "das 2")
        # another output buffer, other flags, another order p, another stream
        out2 = torch.zeros((3, acq.nx, acq.nz), device="cuda")
        bf.bf_beamform(h, rf_d, acq.n_samples, acq.angles_rad, flags | bf.BF_PDAS, out2)
        bf.bf_sync(h)
        p2 = oracle.beamform_pdas(rf2, acq.x_elements(), acq.angles_rad,
                                  (acq.nx, acq.nz, acq.x0_m, acq.x1_m, acq.z0_m, acq.z1_m),
                                  acq.fs_hz, acq.c_mps, acq.f_number, 2.0)
        assert_close(out2.cpu().numpy()[2].astype(np.float64), p2, bf.BF_PREC_FP32, "pdas p=2")
        bf.bf_set_pdas_order(h, 3.0)
        bf.bf_beamform(h, rf_d, acq.n_samples, acq.angles_rad, flags | bf.BF_PDAS, out2)
        bf.bf_sync(h)
        p3 = oracle.beamform_pdas(rf2, acq.x_elements(), acq.angles_rad,
                                  (acq.nx, acq.nz, acq.x0_m, acq.x1_m, acq.z0_m, acq.z1_m),
                                  acq.fs_hz, acq.c_mps, acq.f_number, 3.0)
        assert_close(out2.cpu().numpy()[2].astype(np.float64), p3, bf.BF_PREC_FP32, "pdas p=3")
        s = torch.cuda.Stream()
        bf.bf_set_stream(h, s)
        for _ in range(3):
            out.zero_()
            torch.cuda.synchronize()
            bf.bf_beamform(h, rf_d, acq.n_samples, acq.angles_rad, flags, out)
            s.synchronize()
            assert_close(out.cpu().numpy()[1].astype(np.float64), ref2["dmas"], bf.BF_PREC_FP32,
                         "dmas on a user stream")
        # other angles (another plan) on the same buffers
        bf.bf_beamform(h, rf_d, acq.n_samples, acq.angles_rad[::-1].copy(), flags, out)
        s.synchronize()
        swapped = oracle.beamform(rf2, acq.x_elements(), acq.angles_rad[::-1].copy(),
                                  (acq.nx, acq.nz, acq.x0_m, acq.x1_m, acq.z0_m, acq.z1_m),
                                  acq.fs_hz, acq.c_mps, acq.f_number)
        got = out.cpu().numpy().astype(np.float64)
        # record a is read with angle a of the call
        assert_close(got[0], swapped["das"], bf.BF_PREC_FP32, "reversed angles, records as given")
        bf.bf_set_stream(h, None)
    finally:
        bf.bf_destroy(h)
