"""Stage timing of a batch graph (bf_batch_timing).  The four marks are event
nodes on a side branch of the captured graph, each behind the stage it closes
with no kernel waiting on it: every stage time is positive, the three add up
to no more than the replay timed around the graph launch, and replays with
the marks give the images of the frames beamformed alone (within 0.01 dB: a
multi-frame job sums the DMAS terms' squares where a single frame sums their
magnitudes, which rounds differently)."""
import numpy as np
import pytest

import paper_2311_00482_gb300 as bf
import synth
from test_gpu_parity import make_handle, run_gpu

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


def test_stage_times_positive_and_within_the_replay(torch):
    acq = synth.SPECKLE_POINTS_128.with_(nx=96, nz=128)
    rng = np.random.default_rng(21)
    flags = bf.BF_DAS | bf.BF_DMAS | bf.BF_OUT_LOGDB
    h = make_handle(acq)
    try:
        rfs = [rng.integers(-20000, 20000, (1, acq.n_elements, acq.n_samples)).astype(np.int16)
               for _ in range(6)]
        rf_d = [torch.from_numpy(r).cuda() for r in rfs]
        outs = [torch.zeros((2, acq.nx, acq.nz), device="cuda") for _ in rfs]
        batch = bf.Batch([(h, rf_d[k], acq.n_samples, acq.angles_rad, flags, outs[k])
                          for k in range(len(rfs))])
        try:
            stream = torch.cuda.current_stream()
            for _ in range(4):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                batch.launch(stream)
                b.record(stream)
                b.synchronize()
                ms3, launches = batch.timing()
                step = a.elapsed_time(b)
                assert len(ms3) == 3 and all(t > 0.0 for t in ms3), ms3
                assert sum(ms3) <= step + 1e-3, (ms3, step)
                assert launches >= 4  # ingest, beamform, envelope, log
            batch.status(stream)
        finally:
            batch.close()
        for k in range(len(rfs)):
            np.testing.assert_allclose(outs[k].cpu().numpy().astype(np.float64),
                                       run_gpu(torch, acq, rfs[k], flags, h=h), rtol=0, atol=0.01)
    finally:
        bf.bf_destroy(h)
