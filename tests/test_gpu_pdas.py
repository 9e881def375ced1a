"""pDAS (Eq. (2)-(3)) on the GPU against the FP64 oracle.

Same tolerances as the other combiners (rel-L2 1e-5 FP32, 2e-3 FP16/BF16
storage, per pixel 2e-5 / 1e-2 of the peak).  The p-th power at the end
multiplies a relative error of the compressed sum by p, so the FP16 / BF16
cases stay at p <= 3.
"""
import numpy as np
import pytest

import oracle
import paper_2311_00482_gb300 as bf
import synth
from test_gpu_parity import assert_close, grid_of, make_handle, oracle_all, run_gpu

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


def pdas_ref(acq, rf, p):
    return oracle.beamform_pdas(rf, acq.x_elements(), acq.angles_rad, grid_of(acq), acq.fs_hz,
                                acq.c_mps, acq.f_number, p)


def run_pdas(torch, acq, rf, flags, p):
    h = make_handle(acq)
    try:
        bf.bf_set_pdas_order(h, p)
        return run_gpu(torch, acq, rf, flags, h=h)
    finally:
        bf.bf_destroy(h)


@pytest.mark.parametrize("prec", [bf.BF_PREC_FP32, bf.BF_PREC_FP16, bf.BF_PREC_BF16])
@pytest.mark.parametrize("p", [2.0, 3.0])
def test_ragged_grid_all_four_combiners(torch, prec, p):
    acq = synth.SPECKLE_POINTS_128.with_(nx=100, nz=77, angles_deg=(-6.0, 0.0, 6.0))
    rf, _ = synth.speckle_points_frame(acq)
    ref = oracle_all(acq, rf)
    ref["pdas"] = pdas_ref(acq, rf, p)
    got = run_pdas(torch, acq, rf, bf.BF_DAS | bf.BF_DMAS | bf.BF_CF | bf.BF_PDAS | prec, p)
    assert got.shape[0] == 4
    for k, name in enumerate(("das", "dmas", "cf", "pdas")):
        assert_close(got[k], ref[name], prec, "%s p=%g" % (name, p))


@pytest.mark.parametrize("p", [1.0, 1.5, 2.0, 4.0])
def test_pdas_alone_full_size_and_orders(torch, p):
    acq = synth.CYST_WIRES_512.with_(nx=160, nz=300)
    rf, _ = synth.cyst_wires_frame(acq)
    got = run_pdas(torch, acq, rf, bf.BF_PDAS, p)
    assert got.shape[0] == 1
    assert_close(got[0], pdas_ref(acq, rf, p), bf.BF_PREC_FP32, "pdas p=%g" % p)
    if p == 1.0:  # no compression: the DAS image
        das = run_gpu(torch, acq, rf, bf.BF_DAS)
        np.testing.assert_allclose(got[0], das[0], rtol=0, atol=2e-5 * np.max(np.abs(das[0])))


def test_pdas_plain_kernel_and_envelope(torch):
    acq = synth.SPECKLE_POINTS_128.with_(nx=64, nz=150, angles_deg=(-4.0, 4.0))
    rf, _ = synth.speckle_points_frame(acq)
    ref = pdas_ref(acq, rf, 2.0)
    h = make_handle(acq)
    try:
        rf_d = torch.from_numpy(rf).cuda()
        out = torch.full((1, acq.nx, acq.nz), float("nan"), device="cuda")
        bf.bf_beamform_plain(h, rf_d, acq.n_samples, acq.angles_rad, bf.BF_PDAS, out)
        bf.bf_sync(h)
        assert_close(out.cpu().numpy()[0].astype(np.float64), ref, bf.BF_PREC_FP32, "plain pdas")
        env = run_gpu(torch, acq, rf, bf.BF_PDAS | bf.BF_OUT_ENV, h=h)[0]
        assert_close(env, oracle.envelope(ref), bf.BF_PREC_FP32, "pdas envelope")
        db = run_gpu(torch, acq, rf, bf.BF_PDAS | bf.BF_OUT_LOGDB, h=h)[0]
        assert np.max(np.abs(db - oracle.log_compress(oracle.envelope(ref)))) <= 0.05
    finally:
        bf.bf_destroy(h)


def test_pdas_order_bounds(torch):
    acq = synth.SPECKLE_POINTS_128.with_(nx=8, nz=8)
    h = make_handle(acq)
    try:
        for bad in (0.5, 0.0, -2.0, 17.0, float("nan")):
            with pytest.raises(bf.BFError):
                bf.bf_set_pdas_order(h, bad)
        bf.bf_set_pdas_order(h, 16.0)
    finally:
        bf.bf_destroy(h)
