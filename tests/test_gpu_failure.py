"""Failure paths on the GPU, made without a GPU fault.

A device-side bounded wait that nothing completes runs out and reports
BF_ETIMEDOUT (the path a beamforming CTA whose copies never land takes), and
host-side injected failures (BF_FAULT=alloc|submit|copy) return their codes.
After each, the CUDA context, the handle and the serving engine keep working
and results still match the FP64 oracle.
"""
import numpy as np
import pytest

import paper_2311_00482_gb300 as bf
import synth
from test_gpu_parity import assert_close, make_handle, oracle_all, run_gpu

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


@pytest.fixture(scope="module")
def case():
    acq = synth.SPECKLE_POINTS_128.with_(nx=40, nz=52, angles_deg=(-3.0, 3.0))
    rf, _ = synth.speckle_points_frame(acq, seed=synth.BASE_SEED + 610)
    return acq, rf, oracle_all(acq, rf)


def test_bounded_wait_runs_out_and_the_context_stays_usable(torch, case):
    acq, rf, ref = case
    with pytest.raises(bf.BFError) as ei:
        bf.bf_selftest_wait(2000)  # 2 ms on the device's global timer
    assert ei.value.code == bf.BF_ETIMEDOUT
    for bad in (0, 1_000_001):
        with pytest.raises(bf.BFError) as ei:
            bf.bf_selftest_wait(bad)
        assert ei.value.code == bf.BF_EINVAL
    got = run_gpu(torch, acq, rf, bf.BF_DAS | bf.BF_DMAS)
    assert_close(got[0], ref["das"], bf.BF_PREC_FP32, "das after the timeout")
    assert_close(got[1], ref["dmas"], bf.BF_PREC_FP32, "dmas after the timeout")


def test_injected_allocation_failure_then_recovery(torch, case, monkeypatch):
    acq, rf, ref = case
    h = make_handle(acq)  # the handle's own tables are allocated before the fault
    try:
        monkeypatch.setenv("BF_FAULT", "alloc")
        with pytest.raises(bf.BFError) as ei:
            run_gpu(torch, acq, rf, bf.BF_DAS, h=h)  # the first frame needs a plan
        assert ei.value.code == bf.BF_ENOMEM
        monkeypatch.delenv("BF_FAULT")
        got = run_gpu(torch, acq, rf, bf.BF_DAS, h=h)
        assert_close(got[0], ref["das"], bf.BF_PREC_FP32, "das after an allocation failure")
    finally:
        bf.bf_destroy(h)


def test_injected_admission_and_copy_failures_then_recovery(torch, case, monkeypatch):
    acq, rf, ref = case
    flags = bf.BF_DAS | bf.BF_DMAS
    h = make_handle(acq)
    try:
        rf_host = np.ascontiguousarray(rf)
        # a new handle: its first request must build the plan (device allocations)
        for kind, code in (("alloc", bf.BF_ENOMEM), ("submit", bf.BF_EAGAIN),
                           ("copy", bf.BF_ECUDA), ("alloc,submit", bf.BF_EAGAIN)):
            monkeypatch.setenv("BF_FAULT", kind)
            for _ in range(3):  # repeated refusals leave no request or slot behind
                with pytest.raises(bf.BFError) as ei:
                    bf.bf_submit(h, rf_host, acq.n_samples, acq.angles_rad, flags)
                assert ei.value.code == code, kind
        monkeypatch.delenv("BF_FAULT")
        tickets = [bf.bf_submit(h, rf_host, acq.n_samples, acq.angles_rad, flags) for _ in range(2)]
        for t in tickets:
            out = np.empty((2, acq.nx, acq.nz), np.float32)
            assert bf.bf_poll(h, t, out, timeout_us=30_000_000) == bf.BF_OK
            assert_close(out[0].astype(np.float64), ref["das"], bf.BF_PREC_FP32, "das after faults")
            assert_close(out[1].astype(np.float64), ref["dmas"], bf.BF_PREC_FP32, "dmas after faults")
    finally:
        bf.bf_destroy(h)
