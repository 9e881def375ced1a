"""GPU path (through the C ABI) against the FP64 oracle, element by element.

Tolerances (relative L2 over the image, plus a per-pixel bound relative to the
image's peak): FP32 path 1e-5 / 2e-5; FP16 and BF16 storage 2e-3 / 1e-2.
Envelopes use the same bounds; log-compressed images are compared in dB with
a max-abs bound of 0.05 dB, which is what a 2e-6-of-peak envelope error
becomes at the -70 dB floor (8.7 dB per unit relative error at 3.2e-4 of peak).
"""
import os

import numpy as np
import pytest

import oracle
import paper_2311_00482_gb300 as bf
import synth

pytestmark = pytest.mark.gpu

TOL = {bf.BF_PREC_FP32: (1e-5, 2e-5), bf.BF_PREC_FP16: (2e-3, 1e-2), bf.BF_PREC_BF16: (2e-3, 1e-2)}
MODES = (("das", bf.BF_DAS), ("dmas", bf.BF_DMAS), ("cf", bf.BF_CF))


@pytest.fixture(scope="module")
def torch():
    import torch

    from paper_2311_00482_gb300 import build as bfbuild

    bfbuild.build()
    bf.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    return torch


def grid_of(acq):
    return (acq.nx, acq.nz, acq.x0_m, acq.x1_m, acq.z0_m, acq.z1_m)


def make_handle(acq):
    return bf.bf_create(acq.n_elements, acq.pitch_m, acq.f_number, grid_of(acq), acq.fs_hz,
                        acq.f0_hz, acq.c_mps)


def run_gpu(torch, acq, rf, flags, angles=None, h=None):
    own = h is None
    h = make_handle(acq) if own else h
    try:
        rf_d = torch.from_numpy(np.ascontiguousarray(rf)).cuda()
        nm = bf.n_modes(flags)
        out = torch.full((nm, acq.nx, acq.nz), float("nan"), dtype=torch.float32, device="cuda")
        bf.bf_beamform(h, rf_d, rf.shape[2], acq.angles_rad if angles is None else angles, flags, out)
        bf.bf_sync(h)
        return out.cpu().numpy().astype(np.float64)
    finally:
        if own:
            bf.bf_destroy(h)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def assert_close(got, ref, prec, what):
    l2, elem = TOL[prec]
    assert np.all(np.isfinite(got)), what
    err = rel_l2(got, ref)
    peak = float(np.max(np.abs(ref)))
    worst = float(np.max(np.abs(got - ref)))
    assert err <= l2, "%s: rel-L2 %.3e > %.1e" % (what, err, l2)
    assert worst <= elem * peak, "%s: max abs err %.3e > %.1e of peak" % (what, worst / peak, elem)


def oracle_all(acq, rf):
    return oracle.beamform(rf, acq.x_elements(), acq.angles_rad, grid_of(acq), acq.fs_hz,
                           acq.c_mps, acq.f_number)


# ------------------------------------------------------------ RF stage --

@pytest.mark.parametrize("prec", [bf.BF_PREC_FP32, bf.BF_PREC_FP16, bf.BF_PREC_BF16])
def test_ragged_grid_all_combiners(torch, prec):
    """100 x 77 pixels: 12.5 tiles across, 1.2 tiles deep; record ends inside the field."""
    acq = synth.SPECKLE_POINTS_128.with_(nx=100, nz=77, angles_deg=(-6.0, 0.0, 6.0))
    rf, _ = synth.speckle_points_frame(acq)
    ref = oracle_all(acq, rf)
    got = run_gpu(torch, acq, rf, bf.BF_DAS | bf.BF_DMAS | bf.BF_CF | prec)
    for k, (name, _) in enumerate(MODES):
        assert_close(got[k], ref[name], prec, name)


@pytest.mark.parametrize("flags", [bf.BF_DAS, bf.BF_DMAS, bf.BF_CF, bf.BF_DAS | bf.BF_CF,
                                   bf.BF_DMAS | bf.BF_CF])
def test_mode_subsets_keep_bit_order(torch, flags):
    acq = synth.SPECKLE_POINTS_128.with_(nx=24, nz=70)
    rf, _ = synth.speckle_points_frame(acq)
    ref = oracle_all(acq, rf)
    got = run_gpu(torch, acq, rf, flags)
    names = [n for n, b in MODES if flags & b]
    assert got.shape[0] == len(names)
    for k, name in enumerate(names):
        assert_close(got[k], ref[name], bf.BF_PREC_FP32, name)


def test_full_size_512_das_dmas(torch):
    """The 512 x 512, 2048-sample cyst + wire frame, every pixel."""
    acq = synth.CYST_WIRES_512
    rf, _ = synth.cyst_wires_frame(acq)
    ref = oracle_all(acq, rf)
    got = run_gpu(torch, acq, rf, bf.BF_DAS | bf.BF_DMAS)
    assert_close(got[0], ref["das"], bf.BF_PREC_FP32, "das")
    assert_close(got[1], ref["dmas"], bf.BF_PREC_FP32, "dmas")


def test_degenerate_grids_and_geometry(torch):
    rng = np.random.default_rng(5)
    cases = [
        synth.Acquisition(nx=1, nz=50, x0_m=1e-3, x1_m=1e-3),              # one column
        synth.Acquisition(nx=33, nz=1, z0_m=20e-3, z1_m=20e-3),            # one row
        synth.Acquisition(nx=1, nz=1, x0_m=0.0, x1_m=0.0, z0_m=15e-3, z1_m=15e-3),
        synth.Acquisition(n_elements=1, nx=9, nz=65),                      # single element
        synth.Acquisition(nx=17, nz=66, z0_m=0.0, z1_m=3e-3),              # empty apertures at z=0
        synth.Acquisition(nx=20, nz=90, n_samples=300),                    # most samples off-record
        synth.Acquisition(nx=20, nz=64, angles_deg=(-30.0, 30.0), f_number=0.7),
    ]
    for acq in cases:
        rf = rng.integers(-32768, 32767, (len(acq.angles_deg), acq.n_elements, acq.n_samples)).astype(np.int16)
        ref = oracle_all(acq, rf)
        got = run_gpu(torch, acq, rf, bf.BF_DAS | bf.BF_DMAS | bf.BF_CF)
        # White-noise records make single sums cancel (a single element's DMAS is 0 in exact
        # arithmetic and a rounding residual in FP32), so bound every value against the
        # full-scale magnitude of the terms it sums.  A delay error dn moves an interpolated
        # sample by dn * |u[k+1] - u[k]| <= dn * 2^16, i.e. ~1e-7 of 2^15 per term: DAS and
        # CF-DAS (<= 3x the DAS error) get 1e-5 * M * 2^15.  DMAS's signed square root turns
        # a term error e into at most sqrt(e) near zero, so its bound is 2e-3 * M^2 * 2^14.
        # A wrong channel, angle or index moves a term by ~2^15 and stays far outside these.
        m = ref["m"].astype(np.float64)
        bound = {"das": 1e-5 * m * 32768, "cf": 3e-5 * m * 32768, "dmas": 2e-3 * m * m * 16384}
        for k, (name, _) in enumerate(MODES):
            assert np.all(np.abs(got[k] - ref[name]) <= bound[name] + 1e-30), (acq, name)
            if acq.nx * acq.nz >= 64 and np.max(np.abs(ref[name])) > 0:
                assert_close(got[k], ref[name], bf.BF_PREC_FP32, "%s %s" % (acq, name))


# ------------------------------------------------------ envelope / log --

@pytest.mark.parametrize("nz", [128, 150])
def test_envelope_and_log_stages(torch, nz):
    """Power-of-two depth (radix-2) and 150 rows (Bluestein), fine axial sampling."""
    acq = synth.CYST_WIRES_512.with_(nx=40, nz=nz, z0_m=18e-3, z1_m=18e-3 + (nz - 1) * 20e-6)
    rf, _ = synth.cyst_wires_frame(acq)
    ref = oracle_all(acq, rf)
    dz = (acq.z1_m - acq.z0_m) / (acq.nz - 1)
    flags = bf.BF_DAS | bf.BF_DMAS | bf.BF_CF
    env = run_gpu(torch, acq, rf, flags | bf.BF_OUT_ENV)
    db = run_gpu(torch, acq, rf, flags | bf.BF_OUT_LOGDB)
    for k, (name, _) in enumerate(MODES):
        e_ref = oracle.envelope(ref[name], bandpass=(name == "dmas"), dz=dz, c=acq.c_mps,
                                f0=acq.f0_hz)
        assert_close(env[k], e_ref, bf.BF_PREC_FP32, "env " + name)
        d_ref = oracle.log_compress(e_ref)
        assert np.max(np.abs(db[k] - d_ref)) <= 0.05, name


# -------------------------------------------------------------- batch --

def test_batch_of_uneven_frames_matches_single_frames(torch):
    specs = [(64, 96, 1, bf.BF_DAS), (100, 64, 3, bf.BF_DMAS), (37, 150, 5, bf.BF_DAS | bf.BF_CF),
             (80, 80, 2, bf.BF_DAS | bf.BF_DMAS | bf.BF_OUT_LOGDB), (70, 65, 4, bf.BF_DAS | bf.BF_PREC_FP16)]
    rng = np.random.default_rng(9)
    frames, handles, refs, outs, keep = [], [], [], [], []
    try:
        for nx, nz, na, flags in specs:
            acq = synth.CYST_WIRES_512.with_(nx=nx, nz=nz, angles_deg=synth.angles_linspace(na))
            rf = rng.integers(-20000, 20000, (na, 64, acq.n_samples)).astype(np.int16)
            h = make_handle(acq)
            handles.append(h)
            rf_d = torch.from_numpy(rf).cuda()
            out = torch.zeros((bf.n_modes(flags), nx, nz), dtype=torch.float32, device="cuda")
            keep += [rf_d, out]
            frames.append((h, rf_d, acq.n_samples, acq.angles_rad, flags, out))
            refs.append(run_gpu(torch, acq, rf, flags))
            outs.append(out)
        batch = bf.Batch(frames)
        for _ in range(2):  # replaying the graph gives the same result
            batch.launch()
            batch.status()
            for got, ref in zip(outs, refs):
                np.testing.assert_array_equal(got.cpu().numpy(), ref.astype(np.float32))
        batch.close()
    finally:
        for h in handles:
            bf.bf_destroy(h)


# ------------------------------------------------------------ serving --

def test_submit_poll_results_equal_solo_and_batches_overlap(torch):
    """Continuous batching: requests admitted while launches are held ride
    together; with several batches in flight on the engine's streams their
    device execution overlaps; every result equals the same frame beamformed
    alone."""
    rng = np.random.default_rng(21)
    acqs, rfs, flagss, handles = [], [], [], []
    for k in range(16):
        n = int(rng.integers(64, 200))
        na = int(rng.integers(1, 5))
        acq = synth.CYST_WIRES_512.with_(nx=n, nz=n, angles_deg=synth.angles_linspace(na))
        acqs.append(acq)
        rfs.append(rng.integers(-20000, 20000, (na, 64, acq.n_samples)).astype(np.int16))
        flagss.append([bf.BF_DAS, bf.BF_DMAS][k % 2] | bf.BF_OUT_LOGDB)
        handles.append(make_handle(acq))
    try:
        solo = [run_gpu(torch, a, r, f, h=h) for a, r, f, h in zip(acqs, rfs, flagss, handles)]

        def burst(max_batch, max_inflight):
            bf.bf_engine_configure(max_batch, max_inflight, 0)
            bf.bf_engine_pause(True)
            try:
                tickets = [bf.bf_submit(h, r, a.n_samples, a.angles_rad, f)
                           for a, r, f, h in zip(acqs, rfs, flagss, handles)]
            finally:
                bf.bf_engine_pause(False)
            outs, info, times = [], [], []
            for a, f, h, t in zip(acqs, flagss, handles, tickets):
                got = None
                for _ in range(1000000):
                    got = bf.bf_ticket_batch(h, t)
                    if got is not None:
                        break
                info.append(got)
                for _ in range(1000000):
                    tt = bf.bf_ticket_times(h, t)
                    if tt is not None:
                        break
                times.append(tt)
                out = np.empty((bf.n_modes(f), a.nx, a.nz), np.float32)
                assert bf.bf_poll(h, t, out, timeout_us=10_000_000) == bf.BF_OK
                outs.append(out)
            return tickets, outs, info, times

        # all 16 queued while held: launched together (batches of up to 64)
        tickets, outs, info, _ = burst(64, 1)
        assert max(n for _, n in info) > 1, info
        for out, ref in zip(outs, solo):  # (2e-3 dB: frames of one plan may share a job)
            np.testing.assert_allclose(out, ref, atol=2e-3)
        # batches of 4, three in flight on different streams: some run at the same time
        _, outs, info, times = burst(4, 3)
        for out, ref in zip(outs, solo):
            np.testing.assert_allclose(out, ref, atol=2e-3)
        spans = sorted({(bid, t) for (bid, _), t in zip(info, times)})
        overlap = any(spans[i][1][0] < spans[j][1][1] and spans[j][1][0] < spans[i][1][1]
                      for i in range(len(spans)) for j in range(i + 1, len(spans)))
        assert len(spans) >= 2 and overlap, spans
        with pytest.raises(bf.BFError) as ei:
            bf.bf_poll(handles[0], tickets[0], None, 0)
        assert ei.value.code == bf.BF_ENOTFOUND
    finally:
        bf.bf_engine_pause(False)
        bf.bf_engine_configure(64, 3, 0)
        for h in handles:
            bf.bf_destroy(h)


def test_device_pointer_contract(torch):
    acq = synth.Acquisition(nx=8, nz=8)
    h = make_handle(acq)
    try:
        rf = np.zeros((1, 64, acq.n_samples), np.int16)
        out = torch.zeros((1, 8, 8), device="cuda")
        with pytest.raises(bf.BFError) as ei:
            bf.bf_beamform(h, rf, acq.n_samples, [0.0], bf.BF_DAS, out)
        assert ei.value.code == bf.BF_EINVAL
        rf_d = torch.from_numpy(rf).cuda()
        with pytest.raises(bf.BFError) as ei:
            bf.bf_beamform(h, rf_d, acq.n_samples, [2.0], bf.BF_DAS, out)
        assert ei.value.code == bf.BF_EINVAL
        with pytest.raises(bf.BFError) as ei:
            bf.bf_beamform(h, rf_d, acq.n_samples, [0.0], 0, out)
        assert ei.value.code == bf.BF_EINVAL
    finally:
        bf.bf_destroy(h)


# ------------------------------------------------------- staging windows --

def _delays(acq, ix, iz, i, theta):
    """Fractional sample index of a pixel-channel pair (double precision)."""
    xs, zs = oracle.grid_coords(grid_of(acq))
    xp, zp, xi = xs[ix], zs[iz], acq.x_elements()[i]
    kappa = acq.fs_hz / acq.c_mps
    return (xp * np.sin(theta) + zp * np.cos(theta) + np.sqrt((xp - xi) ** 2 + zp ** 2)) * kappa


@pytest.mark.parametrize("shape", [(33, 1), (40, 37), (100, 77)])
def test_every_counted_sample_lies_in_its_tile_window(torch, shape):
    nx, nz = shape
    acq = synth.SPECKLE_POINTS_128.with_(nx=nx, nz=nz, angles_deg=(-6.0, 0.0, 6.0))
    h = make_handle(acq)
    try:
        info = bf.bf_plan_info(h, acq.n_samples, acq.angles_rad, bf.BF_DAS, with_windows=True)
    finally:
        bf.bf_destroy(h)
    valid, _ = bf.bf_host_tables(acq.n_elements, acq.pitch_m, acq.f_number, grid_of(acq), acq.fs_hz,
                                 acq.f0_hz, acq.c_mps, acq.n_samples, acq.angles_rad)
    th = 8 * info["rows"]
    for a, theta in enumerate(acq.angles_rad):
        for t in range(info["tiles_x"] * info["tiles_z"]):
            tx, tz = t % info["tiles_x"], t // info["tiles_x"]
            for i in range(acq.n_elements):
                w0 = int(info["windows"][a, t, i])
                ks = []
                for ix in range(tx * 32, min(nx, tx * 32 + 32)):
                    lo, hi = valid[a, ix, i]
                    for iz in range(max(lo, tz * th), min(hi, tz * th + th - 1, nz - 1) + 1):
                        ks.append(int(np.floor(_delays(acq, ix, iz, i, theta))))
                if not ks:
                    assert w0 == -2**31, (a, t, i)
                    continue
                # pair j holds samples j - 2 and j - 1: samples k, k + 1 are pair k + 2
                assert w0 <= min(ks) + 2 - 1 and max(ks) + 2 + 1 < w0 + info["wmax"], (a, t, i, w0, min(ks), max(ks))


def test_envelope_into_an_unaligned_output_matches(torch):
    """The envelope stage writes 16-byte vectors only where the destination is
    16-byte aligned; a destination 4 bytes off takes the scalar path, same values."""
    acq = synth.SPECKLE_POINTS_128.with_(nx=40, nz=128)
    rf, _ = synth.speckle_points_frame(acq)
    flags = bf.BF_DAS | bf.BF_DMAS | bf.BF_OUT_ENV
    h = make_handle(acq)
    try:
        rf_d = torch.from_numpy(rf).cuda()
        n = 2 * acq.nx * acq.nz
        aligned = torch.zeros(n, device="cuda")
        big = torch.zeros(n + 1, device="cuda")
        shifted = big[1:]
        assert shifted.data_ptr() % 16 == 4
        bf.bf_beamform(h, rf_d, acq.n_samples, acq.angles_rad, flags, aligned)
        bf.bf_beamform(h, rf_d, acq.n_samples, acq.angles_rad, flags, shifted)
        bf.bf_sync(h)
        np.testing.assert_array_equal(aligned.cpu().numpy(), shifted.cpu().numpy())
        # the log stage too (scalar path into the shifted destination)
        lg = flags & ~bf.BF_OUT_MASK | bf.BF_OUT_LOGDB
        bf.bf_beamform(h, rf_d, acq.n_samples, acq.angles_rad, lg, aligned)
        bf.bf_beamform(h, rf_d, acq.n_samples, acq.angles_rad, lg, shifted)
        bf.bf_sync(h)
        np.testing.assert_array_equal(aligned.cpu().numpy(), shifted.cpu().numpy())
        bf.bf_beamform(h, rf_d, acq.n_samples, acq.angles_rad, flags, aligned)
        bf.bf_sync(h)
        ref = oracle_all(acq, rf)
        dz = (acq.z1_m - acq.z0_m) / (acq.nz - 1)
        env = aligned.cpu().numpy().reshape(2, acq.nx, acq.nz).astype(np.float64)
        assert_close(env[0], oracle.envelope(ref["das"]), bf.BF_PREC_FP32, "das env")
        assert_close(env[1], oracle.envelope(ref["dmas"], bandpass=True, dz=dz, c=acq.c_mps,
                                             f0=acq.f0_hz), bf.BF_PREC_FP32, "dmas env")
    finally:
        bf.bf_destroy(h)


def test_submit_many_and_poll_many(torch):
    """Several frames in one submission and one collection: every result equals
    the frame beamformed alone, from pinned, pageable and device sources into
    pinned, pageable and device destinations."""
    acq = synth.SPECKLE_POINTS_128.with_(nx=48, nz=80)
    flags = bf.BF_DAS | bf.BF_DMAS | bf.BF_OUT_LOGDB
    rfs = [synth.speckle_points_frame(acq, seed=synth.BASE_SEED + 300 + k)[0] for k in range(6)]
    h = make_handle(acq)
    try:
        solo = [run_gpu(torch, acq, rf, flags, h=h) for rf in rfs]
        srcs = [torch.from_numpy(rfs[0]).pin_memory(), rfs[1], torch.from_numpy(rfs[2]).cuda(),
                torch.from_numpy(rfs[3]).pin_memory(), rfs[4], torch.from_numpy(rfs[5]).cuda()]
        tickets = bf.bf_submit_many(h, srcs, acq.n_samples, acq.angles_rad, flags)
        assert len(tickets) == 6 and len(set(tickets)) == 6
        outs = [torch.zeros((2, acq.nx, acq.nz)).pin_memory(), np.zeros((2, acq.nx, acq.nz), np.float32),
                torch.zeros((2, acq.nx, acq.nz), device="cuda"), torch.zeros((2, acq.nx, acq.nz)).pin_memory(),
                np.zeros((2, acq.nx, acq.nz), np.float32), torch.zeros((2, acq.nx, acq.nz), device="cuda")]
        assert bf.bf_poll_many(h, tickets, outs, timeout_us=30_000_000) == bf.BF_OK
        for o, ref in zip(outs, solo):
            got = o if isinstance(o, np.ndarray) else o.cpu().numpy()
            # frames of one plan may ride in a shared multi-frame job (another summation
            # order): 2e-3 dB bounds the rounding difference, 25x below the oracle bound
            np.testing.assert_allclose(got, ref, atol=2e-3)
        with pytest.raises(bf.BFError):  # released
            bf.bf_poll(h, tickets[0], None, timeout_us=0)
    finally:
        bf.bf_destroy(h)


def test_submit_many_and_poll_many_batched_copies(torch):
    """Seventy frames from pinned host records into pinned host images (more
    frames than one batch takes), one image into a destination that is not
    16-byte aligned; every result equals its frame beamformed alone."""
    acq = synth.SPECKLE_POINTS_128.with_(nx=40, nz=64)
    flags = bf.BF_DAS | bf.BF_DMAS
    rfs = [synth.speckle_points_frame(acq, seed=synth.BASE_SEED + 330 + k)[0] for k in range(4)]
    h = make_handle(acq)
    try:
        solo = [run_gpu(torch, acq, rf, flags, h=h) for rf in rfs]
        n = 70
        srcs = [torch.from_numpy(rfs[k % 4]).pin_memory() for k in range(n)]
        size = 2 * acq.nx * acq.nz
        bufs = [torch.full((size + 1,), float("nan")).pin_memory() for _ in range(n)]
        outs = [b[(1 if k == 5 else 0):][:size].view(2, acq.nx, acq.nz) for k, b in enumerate(bufs)]
        tickets = bf.bf_submit_many(h, srcs, acq.n_samples, acq.angles_rad, flags)
        assert bf.bf_poll_many(h, tickets, outs, timeout_us=30_000_000) == bf.BF_OK
        for k, o in enumerate(outs):
            np.testing.assert_allclose(o.numpy(), solo[k % 4], rtol=0,
                                       atol=2e-6 * np.max(np.abs(solo[k % 4])))
    finally:
        bf.bf_destroy(h)


@pytest.mark.parametrize("prec", [bf.BF_PREC_FP32, bf.BF_PREC_FP16])
def test_frames_of_one_plan_share_delays_in_pairs(torch, prec):
    """Five frames of one handle and plan in a batch: two pairs share their delays
    (two-frame jobs), the fifth runs alone; every frame matches the oracle and
    its single-frame result."""
    acq = synth.SPECKLE_POINTS_128.with_(nx=70, nz=90, angles_deg=(-4.0, 4.0))
    flags = bf.BF_DAS | bf.BF_DMAS | prec
    rfs = [synth.speckle_points_frame(acq, seed=synth.BASE_SEED + 500 + k)[0] for k in range(5)]
    h = make_handle(acq)
    try:
        rf_d = [torch.from_numpy(r).cuda() for r in rfs]
        outs = [torch.full((2, acq.nx, acq.nz), float("nan"), device="cuda") for _ in rfs]
        batch = bf.Batch([(h, rf_d[k], acq.n_samples, acq.angles_rad, flags, outs[k])
                          for k in range(5)])
        batch.launch()
        batch.status()
        for k in range(5):
            got = outs[k].cpu().numpy().astype(np.float64)
            ref = oracle_all(acq, rfs[k])
            assert_close(got[0], ref["das"], prec, "das %d" % k)
            assert_close(got[1], ref["dmas"], prec, "dmas %d" % k)
            single = run_gpu(torch, acq, rfs[k], flags, h=h)
            np.testing.assert_allclose(got, single, rtol=0,
                                       atol=2e-6 * np.max(np.abs(single)) + 1e-30)
        batch.close()
    finally:
        bf.bf_destroy(h)


# (precision, depth, output offset in floats): depth 92 with aligned images
# takes the bulk-copy epilogue (ragged last tile), 90 the 8-byte row-pair
# stores, 91 and images offset by one float the per-pixel stores
@pytest.mark.parametrize("prec,nz,offset", [(bf.BF_PREC_FP32, 90, 0), (bf.BF_PREC_FP32, 92, 0),
                                            (bf.BF_PREC_FP32, 91, 0), (bf.BF_PREC_FP32, 92, 1),
                                            (bf.BF_PREC_BF16, 90, 0), (bf.BF_PREC_BF16, 92, 0)])
def test_two_row_tiles_share_delays_in_fours(torch, monkeypatch, prec, nz, offset):
    """Seven frames of one plan on 16-row tiles: one four-frame job, one
    two-frame job and one frame alone; every frame matches the oracle and its
    single-frame result on the same tiles."""
    monkeypatch.setenv("BF_TILE_ROWS", "2")
    acq = synth.SPECKLE_POINTS_128.with_(nx=70, nz=nz, angles_deg=(-4.0, 4.0))
    flags = bf.BF_DAS | bf.BF_DMAS | prec
    rfs = [synth.speckle_points_frame(acq, seed=synth.BASE_SEED + 520 + k)[0] for k in range(7)]
    h = make_handle(acq)
    try:
        assert bf.bf_plan_info(h, acq.n_samples, acq.angles_rad, flags)["rows"] == 2
        rf_d = [torch.from_numpy(r).cuda() for r in rfs]
        n = 2 * acq.nx * acq.nz
        bufs = [torch.full((n + offset,), float("nan"), device="cuda") for _ in rfs]
        outs = [b[offset:].view(2, acq.nx, acq.nz) for b in bufs]
        batch = bf.Batch([(h, rf_d[k], acq.n_samples, acq.angles_rad, flags, outs[k])
                          for k in range(7)])
        batch.launch()
        batch.status()
        for k in range(7):
            got = outs[k].cpu().numpy().astype(np.float64)
            ref = oracle_all(acq, rfs[k])
            assert_close(got[0], ref["das"], prec, "das %d" % k)
            assert_close(got[1], ref["dmas"], prec, "dmas %d" % k)
            single = run_gpu(torch, acq, rfs[k], flags, h=h)
            np.testing.assert_allclose(got, single, rtol=0,
                                       atol=2e-6 * np.max(np.abs(single)) + 1e-30)
        batch.close()
    finally:
        bf.bf_destroy(h)


def test_two_row_tiles_leave_other_combiners_on_the_default(torch, monkeypatch):
    """Two-row tiles carry DAS / DMAS only: a coherence-factor or pDAS frame on a
    handle asked for them keeps the default 32-row tiles and still matches."""
    monkeypatch.setenv("BF_TILE_ROWS", "2")
    acq = synth.SPECKLE_POINTS_128.with_(nx=40, nz=60, angles_deg=(0.0,))
    rf, _ = synth.speckle_points_frame(acq)
    h = make_handle(acq)
    try:
        assert bf.bf_plan_info(h, acq.n_samples, acq.angles_rad, bf.BF_DAS)["rows"] == 2
        flags = bf.BF_DAS | bf.BF_CF
        assert bf.bf_plan_info(h, acq.n_samples, acq.angles_rad, flags)["rows"] == 4
        ref = oracle_all(acq, rf)
        got = run_gpu(torch, acq, rf, flags, h=h)
        assert_close(got[0], ref["das"], bf.BF_PREC_FP32, "das")
        assert_close(got[1], ref["cf"], bf.BF_PREC_FP32, "cf")
    finally:
        bf.bf_destroy(h)


def test_submit_many_into_delivers_to_every_destination_kind(torch):
    """Results delivered by the batches themselves to destinations given at
    submission: pinned, pageable and device buffers; every one equals the
    frame beamformed alone, and polling (without outputs) releases the tickets."""
    acq = synth.SPECKLE_POINTS_128.with_(nx=48, nz=80)
    flags = bf.BF_DAS | bf.BF_DMAS | bf.BF_OUT_LOGDB
    rfs = [synth.speckle_points_frame(acq, seed=synth.BASE_SEED + 360 + k)[0] for k in range(6)]
    h = make_handle(acq)
    try:
        solo = [run_gpu(torch, acq, rf, flags, h=h) for rf in rfs]
        srcs = [torch.from_numpy(rfs[0]).pin_memory(), rfs[1], torch.from_numpy(rfs[2]).cuda(),
                torch.from_numpy(rfs[3]).pin_memory(), rfs[4], torch.from_numpy(rfs[5]).cuda()]
        outs = [torch.full((2, acq.nx, acq.nz), float("nan")).pin_memory(),
                np.full((2, acq.nx, acq.nz), np.nan, np.float32),
                torch.full((2, acq.nx, acq.nz), float("nan"), device="cuda"),
                torch.full((2, acq.nx, acq.nz), float("nan"), device="cuda"),
                torch.full((2, acq.nx, acq.nz), float("nan")).pin_memory(),
                np.full((2, acq.nx, acq.nz), np.nan, np.float32)]
        for _ in range(2):  # the second round reuses the released slots
            tickets = bf.bf_submit_many_into(h, srcs, acq.n_samples, acq.angles_rad, flags, outs)
            assert bf.bf_poll_many(h, tickets, None, timeout_us=30_000_000) == bf.BF_OK
            for o, ref in zip(outs, solo):
                got = o if isinstance(o, np.ndarray) else o.cpu().numpy()
                np.testing.assert_allclose(got, ref, atol=2e-3)
            with pytest.raises(bf.BFError):  # released
                bf.bf_poll(h, tickets[0], None, timeout_us=0)
            for o in outs:
                o.fill_(float("nan")) if not isinstance(o, np.ndarray) else o.fill(np.nan)
        # single polls release such tickets too
        tickets = bf.bf_submit_many_into(h, srcs[:2], acq.n_samples, acq.angles_rad, flags, outs[:2])
        for t in tickets:
            assert bf.bf_poll(h, t, None, timeout_us=30_000_000) == bf.BF_OK
        for o, ref in zip(outs[:2], solo[:2]):
            got = o if isinstance(o, np.ndarray) else o.cpu().numpy()
            np.testing.assert_allclose(got, ref, atol=2e-3)
        # destinations in one buffer (BF_DEST_ONE_BUFFER), host or device:
        # neighbours leave in one transfer per run; a gap splits the run
        for buf in (torch.full((7, 2, acq.nx, acq.nz), float("nan")).pin_memory(),
                    torch.full((7, 2, acq.nx, acq.nz), float("nan"), device="cuda"),
                    np.full((7, 2, acq.nx, acq.nz), np.nan, np.float32)):  # pageable: staged
            views = [buf[k] for k in (0, 1, 2, 4, 5, 6)]  # buf[3] stays untouched
            tickets = bf.bf_submit_many_into(h, srcs, acq.n_samples, acq.angles_rad,
                                             flags | bf.BF_DEST_ONE_BUFFER, views)
            assert bf.bf_poll_many(h, tickets, None, timeout_us=30_000_000) == bf.BF_OK
            for v, ref in zip(views, solo):
                got = v if isinstance(v, np.ndarray) else v.cpu().numpy()
                np.testing.assert_allclose(got, ref, atol=2e-3)
            assert np.isnan(buf[3] if isinstance(buf, np.ndarray) else buf[3].cpu().numpy()).all()
        small = [torch.zeros(4)]
        with pytest.raises(bf.BFError) as ei:
            bf.bf_submit_many_into(h, srcs[:1], acq.n_samples, acq.angles_rad, flags, small)
        assert ei.value.code == bf.BF_EINVAL
    finally:
        bf.bf_destroy(h)


@pytest.mark.parametrize("stage", [bf.BF_OUT_RF, bf.BF_OUT_ENV, bf.BF_OUT_LOGDB])
def test_one_buffer_delivery_for_every_output_stage(torch, stage):
    """bf_submit_many_into with BF_DEST_ONE_BUFFER: the batch's kernels write the
    images (beamformed, envelope or dB) into its result arena and the views of
    one pinned buffer receive them in one transfer; each equals the frame
    beamformed alone, on 16-row tiles (four-frame jobs) as on the default tiles."""
    acq = synth.SPECKLE_POINTS_128.with_(nx=48, nz=96)
    flags = bf.BF_DAS | bf.BF_DMAS | stage
    rfs = [synth.speckle_points_frame(acq, seed=synth.BASE_SEED + 380 + k)[0] for k in range(5)]
    for rows in ("2", None):
        if rows:
            os.environ["BF_TILE_ROWS"] = rows
        h = make_handle(acq)
        try:
            solo = [run_gpu(torch, acq, rf, flags, h=h) for rf in rfs]
            srcs = [torch.from_numpy(r).pin_memory() for r in rfs]
            buf = torch.full((5, 2, acq.nx, acq.nz), float("nan")).pin_memory()
            tickets = bf.bf_submit_many_into(h, srcs, acq.n_samples, acq.angles_rad,
                                             flags | bf.BF_DEST_ONE_BUFFER, list(buf))
            assert bf.bf_poll_many(h, tickets, None, timeout_us=30_000_000) == bf.BF_OK
            for k in range(5):
                # four-frame jobs round the DMAS sums differently from single frames
                # (a few 1e-6 relative: 4e-4 dB near the -70 dB floor); a frame in
                # the wrong place would be off by whole decibels
                atol = 0.01 if stage == bf.BF_OUT_LOGDB else 2e-6 * np.max(np.abs(solo[k]))
                np.testing.assert_allclose(buf[k].numpy(), solo[k], rtol=0, atol=atol + 1e-30)
        finally:
            bf.bf_destroy(h)
            os.environ.pop("BF_TILE_ROWS", None)
