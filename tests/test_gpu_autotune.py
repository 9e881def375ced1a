"""The tile autotuner: it times every configuration, keeps the fastest for the
workload, and results under every configuration still match the oracle."""
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


def test_autotune_choice_is_kept_and_exact(torch, monkeypatch):
    monkeypatch.delenv("BF_TILE_ROWS", raising=False)
    acq = synth.SPECKLE_POINTS_128.with_(nx=100, nz=140, angles_deg=(-5.0, 5.0))
    rf, _ = synth.speckle_points_frame(acq)
    flags = bf.BF_DAS | bf.BF_DMAS | bf.BF_CF
    ref = oracle_all(acq, rf)
    h = make_handle(acq)
    try:
        res = bf.bf_autotune(h, acq.n_samples, acq.angles_rad, flags, frames=4)
        assert res["rows"] in (4, 8)
        assert res["stage_bytes"] in (16 << 10, 24 << 10, 32 << 10)
        times = [t for t in res["candidates_us"] if t > 0]
        assert len(times) >= 2 and min(times) > 0
        info = bf.bf_plan_info(h, acq.n_samples, acq.angles_rad, flags)
        assert info["rows"] == res["rows"]
        got = run_gpu(torch, acq, rf, flags, h=h)
        for k, name in enumerate(("das", "dmas", "cf")):
            assert_close(got[k], ref[name], bf.BF_PREC_FP32, "tuned " + name)
    finally:
        bf.bf_destroy(h)


@pytest.mark.parametrize("rows", ["2", "4", "8"])
def test_every_tile_height_matches_the_oracle(torch, monkeypatch, rows):
    monkeypatch.setenv("BF_TILE_ROWS", rows)
    acq = synth.SPECKLE_POINTS_128.with_(nx=70, nz=101, angles_deg=(0.0, 7.0))
    rf, _ = synth.speckle_points_frame(acq)
    ref = oracle_all(acq, rf)
    h = make_handle(acq)
    try:
        info = bf.bf_plan_info(h, acq.n_samples, acq.angles_rad, bf.BF_DAS)
        assert info["rows"] == int(rows)
        got = run_gpu(torch, acq, rf, bf.BF_DAS | bf.BF_DMAS | bf.BF_PREC_FP16, h=h)
        assert_close(got[0], ref["das"], bf.BF_PREC_FP16, "das rows=" + rows)
        assert_close(got[1], ref["dmas"], bf.BF_PREC_FP16, "dmas rows=" + rows)
    finally:
        bf.bf_destroy(h)


def test_autotune_rejects_bad_frame_counts(torch):
    acq = synth.SPECKLE_POINTS_128.with_(nx=16, nz=16)
    h = make_handle(acq)
    try:
        for frames in (0, 257):
            with pytest.raises(bf.BFError):
                bf.bf_autotune(h, acq.n_samples, acq.angles_rad, bf.BF_DAS, frames=frames)
    finally:
        bf.bf_destroy(h)
