"""The allocation-free entry point bf_logdb_static, for callers that cannot
allocate device memory while running.

A real-time acquisition loop that must not enter cudaMalloc after start-up, or
an application whose device memory belongs to its own allocator, hands the
library a beamformed image it already holds and gets back the -70 dB
log-compressed envelope (the B-mode display of Fig. 3) in its own buffer.
The inputs here are the oracle's own beamformed images (in FP32, as a caller
would hold them); the expected dB images are the oracle's envelope and log
compression of the same images.  The checks:

* every pixel within the first-order effect of an envelope error of 2e-6 of
  A = max(peak envelope, peak |image|) (0.054 dB at the -70 dB floor without a
  band-pass), on two calls in a row (the scratch array keeps the previous
  call's contents), without and with the DMAS band-pass;
* the largest depth the array takes, 4096 rows (256 x 4096 = 2^20 pixels);
* the device's free memory is unchanged across calls (nothing is allocated);
* sizes beyond the array are rejected.

Collected last, so that a run stopping at its first failure has run every
other test first.
"""
import numpy as np
import pytest

import oracle
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


def oracle_case(acq, seed):
    """FP32 DAS / DMAS images of a frame (the caller's input) and the oracle's dB
    images of exactly those FP32 images."""
    rf, _ = synth.cyst_wires_frame(acq, seed=seed)
    grid = (acq.nx, acq.nz, acq.x0_m, acq.x1_m, acq.z0_m, acq.z1_m)
    r = oracle.beamform(rf, acq.x_elements(), acq.angles_rad, grid, acq.fs_hz, acq.c_mps,
                        acq.f_number)
    dz = (acq.z1_m - acq.z0_m) / (acq.nz - 1)
    cases = []
    for name, band in (("das", 0), ("dmas", 1)):
        y = r[name].astype(np.float32)
        env = oracle.envelope(y.astype(np.float64), bandpass=bool(band), dz=dz, c=acq.c_mps,
                              f0=acq.f0_hz)
        cases.append((y, band, env, oracle.log_compress(env)))
    return cases


def check_db(got, env, db, y, what):
    amp = max(float(env.max()), float(np.max(np.abs(y))))
    e = 2e-6 * amp
    peak = float(env.max())
    tol = 8.686 * e / np.maximum(env, 10 ** (-70 / 20) * peak) + 8.686 * e / peak
    assert np.all(np.isfinite(got)), what
    bad = np.abs(got - db) > tol
    assert not bad.any(), "%s: %d pixels off, worst %.4f dB" % (what, int(bad.sum()),
                                                              float(np.max(np.abs(got - db))))


def run_static(torch, acq, cases, repeats=2):
    """bf_logdb_static on each case, `repeats` times in a row; returns the dB
    images of the last round and the device's free memory around the calls
    after the first one."""
    ys = [torch.from_numpy(y).cuda() for y, _, _, _ in cases]
    outs = [torch.full((acq.nx, acq.nz), float("nan"), device="cuda") for _ in cases]
    got, free = [], []
    for rnd in range(repeats):
        for k, (y, band, _, _) in enumerate(cases):
            outs[k].fill_(float("nan"))
            torch.cuda.synchronize()
            if rnd > 0:
                free.append(torch.cuda.mem_get_info()[0])
            bf.bf_logdb_static(ys[k], acq.nx, acq.nz, acq.z0_m, acq.z1_m, acq.f0_hz, acq.c_mps,
                               band, outs[k])
            torch.cuda.synchronize()
            if rnd > 0:
                free.append(torch.cuda.mem_get_info()[0])
        got = [o.cpu().numpy().astype(np.float64) for o in outs]
        for k, (y, band, env, db) in enumerate(cases):
            check_db(got[k], env, db, y, "round %d band %d" % (rnd, band))
    return got, free


def test_static_logdb_matches_the_oracle_twice_and_allocates_nothing(torch):
    acq = synth.CYST_WIRES_512.with_(nx=96, nz=256, z0_m=15e-3, z1_m=15e-3 + 255 * 20e-6)
    cases = oracle_case(acq, synth.BASE_SEED + 800)
    _, free = run_static(torch, acq, cases, repeats=3)
    assert len(set(free)) == 1, "device memory changed across calls: %s" % free


def test_static_logdb_at_the_largest_depth(torch):
    acq = synth.CYST_WIRES_512.with_(nx=256, nz=4096, x0_m=-3.84e-3, x1_m=3.84e-3,
                                     z0_m=12e-3, z1_m=12e-3 + 4095 * 5e-6)
    cases = oracle_case(acq, synth.BASE_SEED + 801)
    _, free = run_static(torch, acq, cases, repeats=2)
    assert len(set(free)) == 1, "device memory changed across calls: %s" % free


def test_static_logdb_rejects_sizes_beyond_its_array(torch):
    y = torch.zeros((2048, 1024), dtype=torch.float32, device="cuda")
    with pytest.raises(bf.BFError) as ei:  # 2^21 pixels
        bf.bf_logdb_static(y, 2048, 1024, 5e-3, 40e-3, 5e6, 1540.0, 0, y)
    assert ei.value.code == bf.BF_EINVAL
    with pytest.raises(bf.BFError) as ei:  # depth beyond 4096
        bf.bf_logdb_static(y, 128, 8192, 5e-3, 40e-3, 5e6, 1540.0, 0, y)
    assert ei.value.code == bf.BF_EINVAL
    with pytest.raises(bf.BFError) as ei:  # not a power of two
        bf.bf_logdb_static(y, 16, 300, 5e-3, 40e-3, 5e6, 1540.0, 0, y)
    assert ei.value.code == bf.BF_EINVAL
