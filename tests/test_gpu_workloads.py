"""Full-size workloads on the GPU against the FP64 oracle.

* plain baseline kernel (one frame per launch) vs the oracle;
* the uneven 256-frame batch (grids 64..1024 pixels per side, 1..11 angles,
  2048 samples, DAS and DMAS) in one CUDA-graph launch, on pixels sampled from
  every frame (the oracle computes them one by one);
* the precision workload (1024 x 1024, 128 elements, 4096 samples, 7 angles)
  with FP32, FP16 and BF16 storage: relative L2 on sampled pixels, and CNR
  (dB) / FWHM deltas against the oracle on the columns around the cyst;
* a Poisson-timed serving trace with FP16 storage: every result equals the
  same frame beamformed alone.
"""
import math
import time

import numpy as np
import pytest

import oracle
import paper_2311_00482_gb300 as bf
import synth
from test_gpu_parity import TOL, assert_close, grid_of, make_handle, oracle_all, rel_l2, run_gpu

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


def test_plain_kernel_matches_oracle_and_tiled_path(torch):
    acq = synth.SPECKLE_POINTS_128.with_(nx=100, nz=77, angles_deg=(-6.0, 0.0, 6.0))
    rf, _ = synth.speckle_points_frame(acq)
    ref = oracle_all(acq, rf)
    flags = bf.BF_DAS | bf.BF_DMAS | bf.BF_CF
    h = make_handle(acq)
    try:
        rf_d = torch.from_numpy(rf).cuda()
        out = torch.full((3, acq.nx, acq.nz), float("nan"), device="cuda")
        bf.bf_beamform_plain(h, rf_d, acq.n_samples, acq.angles_rad, flags, out)
        db = torch.full((3, acq.nx, acq.nz), float("nan"), device="cuda")
        bf.bf_beamform_plain(h, rf_d, acq.n_samples, acq.angles_rad, flags | bf.BF_OUT_LOGDB, db)
        bf.bf_sync(h)
        got = out.cpu().numpy().astype(np.float64)
        for k, name in enumerate(("das", "dmas", "cf")):
            assert_close(got[k], ref[name], bf.BF_PREC_FP32, "plain " + name)
        tiled = run_gpu(torch, acq, rf, flags | bf.BF_OUT_LOGDB, h=h)
        assert np.max(np.abs(db.cpu().numpy() - tiled)) <= 0.05
        with pytest.raises(bf.BFError):
            bf.bf_beamform_plain(h, rf_d, acq.n_samples, acq.angles_rad, flags | bf.BF_PREC_FP16, out)
    finally:
        bf.bf_destroy(h)


def test_uneven_256_frame_batch_sampled_against_oracle(torch):
    specs = synth.mixed_batch_specs(256)
    rng = np.random.default_rng(synth.BASE_SEED + 2)
    frames, handles, keep, meta = [], [], [], []
    try:
        for k, sp in enumerate(specs):
            na = sp["n_angles"]
            acq = synth.CYST_WIRES_512.with_(nx=sp["nx"], nz=sp["nz"],
                                             angles_deg=synth.angles_linspace(na))
            rf = rng.integers(-20000, 20000, (na, 64, acq.n_samples)).astype(np.int16)
            flags = bf.BF_DAS if k % 2 == 0 else bf.BF_DMAS
            h = make_handle(acq)
            handles.append(h)
            rf_d = torch.from_numpy(rf).cuda()
            out = torch.zeros((1, acq.nx, acq.nz), dtype=torch.float32, device="cuda")
            keep += [rf_d, out]
            frames.append((h, rf_d, acq.n_samples, acq.angles_rad, flags, out))
            meta.append((acq, rf, flags, out))
        batch = bf.Batch(frames)
        batch.launch()
        batch.status()
        got_all, ref_all = [], []
        for acq, rf, flags, out in meta:
            n = 48
            pix = rng.integers(0, acq.nx * acq.nz, n)
            r = oracle.beamform(rf, acq.x_elements(), acq.angles_rad, grid_of(acq), acq.fs_hz,
                                acq.c_mps, acq.f_number, pixels=pix)
            name = "das" if flags == bf.BF_DAS else "dmas"
            got = out.cpu().numpy().reshape(-1)[pix].astype(np.float64)
            got_all.append(got / np.sqrt(np.mean(r[name] ** 2) + 1e-30))
            ref_all.append(r[name] / np.sqrt(np.mean(r[name] ** 2) + 1e-30))
        got_all, ref_all = np.concatenate(got_all), np.concatenate(ref_all)
        assert rel_l2(got_all, ref_all) <= 1e-5
        # a few frames again through bf_beamform: identical to their batch result
        for acq, rf, flags, out in meta[:6]:
            single = run_gpu(torch, acq, rf, flags)
            np.testing.assert_array_equal(single.astype(np.float32), out.cpu().numpy())
        batch.close()
    finally:
        for h in handles:
            bf.bf_destroy(h)


@pytest.fixture(scope="module")
def precision_case():
    acq = synth.PRECISION_1024
    rf, ph = synth.precision_frame(acq)
    # oracle on the columns around the cyst (0, 17.5 mm, r = 2 mm) and its side regions
    xs, zs = oracle.grid_coords(grid_of(acq))
    cols = np.nonzero(np.abs(xs) <= 7.5e-3)[0]
    pix = (cols[:, None] * acq.nz + np.arange(acq.nz)[None, :]).reshape(-1)
    ref = oracle.beamform(rf, acq.x_elements(), acq.angles_rad, grid_of(acq), acq.fs_hz,
                          acq.c_mps, acq.f_number, pixels=pix)
    ref = {k: v.reshape(len(cols), acq.nz) for k, v in ref.items()}
    return acq, rf, cols, ref


@pytest.mark.parametrize("prec", [bf.BF_PREC_FP32, bf.BF_PREC_FP16, bf.BF_PREC_BF16])
def test_precision_workload_l2_cnr_fwhm(torch, precision_case, prec):
    acq, rf, cols, ref = precision_case
    flags = bf.BF_DAS | bf.BF_DMAS | bf.BF_CF | prec
    got = run_gpu(torch, acq, rf, flags)[:, cols, :]
    dz = (acq.z1_m - acq.z0_m) / (acq.nz - 1)
    xs, zs = oracle.grid_coords(grid_of(acq))
    sub = (len(cols), acq.nz, xs[cols[0]], xs[cols[-1]], acq.z0_m, acq.z1_m)
    inside, outside = oracle.cyst_regions(sub, 0.0, 17.5e-3, 2e-3)
    l2, _ = TOL[prec]
    for k, name in enumerate(("das", "dmas", "cf")):
        assert rel_l2(got[k], ref[name]) <= l2, (name, rel_l2(got[k], ref[name]))
        bp = name == "dmas"
        e_ref = oracle.envelope(ref[name], bandpass=bp, dz=dz, c=acq.c_mps, f0=acq.f0_hz)
        e_got = oracle.envelope(got[k], bandpass=bp, dz=dz, c=acq.c_mps, f0=acq.f0_hz)
        c_ref = oracle.contrast(e_ref, inside, outside)
        c_got = oracle.contrast(e_got, inside, outside)
        assert abs(20 * math.log10(c_got["cnr"]) - 20 * math.log10(c_ref["cnr"])) <= 0.1, name
        # wire at (0, 12 mm): lateral and axial FWHM within one pixel
        ix = int(np.argmin(np.abs(xs[cols] - 0.0)))
        iz0 = int(np.argmin(np.abs(zs - 12e-3)))
        win = slice(iz0 - 40, iz0 + 41)
        iz = iz0 - 40 + int(np.argmax(e_ref[ix, win]))
        dx = xs[1] - xs[0]
        assert abs(oracle.fwhm(e_got[:, iz], dx) - oracle.fwhm(e_ref[:, iz], dx)) <= dx, name
        assert abs(oracle.fwhm(e_got[ix, win], dz) - oracle.fwhm(e_ref[ix, win], dz)) <= dz, name


def test_poisson_serving_trace_fp16(torch):
    """Requests of random grids 128..1024, 1..7 angles, DAS or DMAS, FP16 storage,
    arriving as a Poisson process at 2 kHz: every result equals the frame alone."""
    rng = np.random.default_rng(synth.BASE_SEED + 4)
    pool = [rng.integers(-20000, 20000, (7, 64, 2048)).astype(np.int16) for _ in range(4)]
    reqs, handles = [], {}
    for k in range(40):
        n = int(rng.integers(128, 1025))
        na = int(rng.integers(1, 8))
        acq = synth.CYST_WIRES_512.with_(nx=n, nz=n, angles_deg=synth.angles_linspace(na))
        flags = (bf.BF_DAS if rng.random() < 0.5 else bf.BF_DMAS) | bf.BF_PREC_FP16 | bf.BF_OUT_LOGDB
        rf = np.ascontiguousarray(pool[k % 4][:na])
        h = make_handle(acq)
        handles[k] = h
        reqs.append((acq, rf, flags, h))
    try:
        solo = [run_gpu(torch, a, r, f, h=h) for a, r, f, h in reqs]
        gaps = rng.exponential(1.0 / 2000.0, len(reqs))
        tickets = []
        t_next = time.perf_counter()
        for (a, r, f, h), g in zip(reqs, gaps):
            t_next += g
            while time.perf_counter() < t_next:
                pass
            while True:
                try:
                    tickets.append(bf.bf_submit(h, r, a.n_samples, a.angles_rad, f))
                    break
                except bf.BFError as e:  # admission refused: retry once memory frees up
                    assert e.code == bf.BF_EAGAIN
                    time.sleep(1e-4)
        for (a, r, f, h), t, ref in zip(reqs, tickets, solo):
            out = np.empty((1, a.nx, a.nz), np.float32)
            assert bf.bf_poll(h, t, out, timeout_us=30_000_000) == bf.BF_OK
            # requests of one plan may share a multi-frame job (another summation order)
            np.testing.assert_allclose(out, ref, atol=2e-3)
    finally:
        for h in handles.values():
            bf.bf_destroy(h)
