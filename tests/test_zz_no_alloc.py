"""The allocation-free entry point bf_logdb_static, for callers that cannot
allocate device memory while running, against the regular path.

bf_beamform computes the beamformed images (BF_OUT_RF) and, separately, their
log-compressed envelopes (BF_OUT_LOGDB).  bf_logdb_static, fed the beamformed
images, must return the same decibel images within the 0.05 dB bound the
other log-compression tests use, on two calls in a row (its scratch array is
reused and keeps the previous call's contents).  Collected last so that a run
stopping at the first failure has run every other test first.
"""
import numpy as np
import pytest

import paper_2311_00482_gb300 as bf
import synth

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


def test_static_logdb_matches_regular_path_twice(torch):
    acq = synth.CYST_WIRES_512.with_(nx=96, nz=256, z0_m=15e-3, z1_m=15e-3 + 255 * 20e-6)
    rf, _ = synth.cyst_wires_frame(acq)
    grid = (acq.nx, acq.nz, acq.x0_m, acq.x1_m, acq.z0_m, acq.z1_m)
    h = bf.bf_create(acq.n_elements, acq.pitch_m, acq.f_number, grid, acq.fs_hz, acq.f0_hz,
                     acq.c_mps)
    try:
        rf_d = torch.from_numpy(rf).cuda()
        modes = bf.BF_DAS | bf.BF_DMAS
        y = torch.empty((2, acq.nx, acq.nz), dtype=torch.float32, device="cuda")
        ref = torch.empty_like(y)
        bf.bf_beamform(h, rf_d, acq.n_samples, acq.angles_rad, modes | bf.BF_OUT_RF, y)
        bf.bf_beamform(h, rf_d, acq.n_samples, acq.angles_rad, modes | bf.BF_OUT_LOGDB, ref)
        bf.bf_sync(h)
        ref = ref.cpu().numpy()
        for _ in range(2):  # DAS (no band-pass) then DMAS (band-pass), twice
            for k, band in ((0, 0), (1, 1)):
                out = torch.full((acq.nx, acq.nz), float("nan"), dtype=torch.float32, device="cuda")
                bf.bf_logdb_static(y[k], acq.nx, acq.nz, acq.z0_m, acq.z1_m, acq.f0_hz, acq.c_mps,
                                   band, out)
                torch.cuda.synchronize()
                got = out.cpu().numpy()
                assert np.all(np.isfinite(got))
                assert np.max(np.abs(got - ref[k])) <= 0.05, (k, np.max(np.abs(got - ref[k])))
    finally:
        bf.bf_destroy(h)


def test_static_logdb_rejects_sizes_beyond_its_array(torch):
    y = torch.zeros((2048, 1024), dtype=torch.float32, device="cuda")
    with pytest.raises(bf.BFError) as ei:
        bf.bf_logdb_static(y, 2048, 1024, 5e-3, 40e-3, 5e6, 1540.0, 0, y)
    assert ei.value.code == bf.BF_EINVAL
    with pytest.raises(bf.BFError) as ei:
        bf.bf_logdb_static(y, 16, 300, 5e-3, 40e-3, 5e6, 1540.0, 0, y)  # not a power of two
    assert ei.value.code == bf.BF_EINVAL
