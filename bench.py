#!/usr/bin/env python3
"""Throughput / latency benchmark of the plane-wave beamformer.

Workload (one step): a batch of B frames of the 512 x 512-pixel cyst + wire
acquisition (64 receive channels, 2048 int16 samples, one 0 deg plane wave,
5 MHz, 20 MHz sampling), each through the whole path: RF ingest, DAS and
signed-sqrt DMAS beamforming, envelope (DMAS through its 2 f0 band-pass) and
-70 dB log compression.  Inputs are synthetic (seeded phantoms standing in
for the paper's PVA phantom recordings).

Legs:
  device  the batch is a captured CUDA graph replayed on device-resident RF;
          L2 is flushed (256 MiB write) before every timed step; the step and
          the beamforming kernels are timed with events captured in the graph
  e2e     the same frames through bf_submit / bf_poll with pinned host RF and
          host outputs (host -> device and device -> host copies timed); per
          frame submit-to-result latency gives p50 / p99
  cpu     the FP64 oracle on the host cores, a bounded sample of frames

--impl reference times the oracle alone (the method as the paper states it,
on the CPU) with the same metric; with torchrun only rank 0 runs it.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

# steps the end-to-end leg keeps in flight
E2E_DEPTH = 2

METRIC = "Gpixel*ch/s (DAS+DMAS 512^2 x 64ch, envelope + log), frames/s, p50/p99 frame latency"
UNIT = "Gpixel*ch/s"
WORKLOAD = ("cyst+wires phantom, 512x512 pixels, 64 ch, 2048 int16 samples, 1 plane wave (0 deg), "
            "DAS+DMAS, Hilbert envelope (DMAS 2f0 band-pass), -70 dB log")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--frames", type=int, default=64, help="frames per step")
    p.add_argument("--prec", default="fp32", choices=["fp32", "fp16", "bf16"])
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-serving", action="store_true", help="skip the short serving-latency leg")
    p.add_argument("--no-tune", action="store_true",
                   help="skip the autotuner: the library's default tiles, or BF_TILE_ROWS (profiling)")
    p.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling)")
    p.add_argument("--workload", default="cyst512",
                   choices=["cyst512", "batch256", "serving", "precision", "sweep", "iq", "fk"],
                   help="cyst512: the headline line; the others print informational lines")
    p.add_argument("--requests", type=int, default=2000, help="serving: requests per rate")
    return p.parse_args()


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# DRAM bytes (read + write) of one beamform_kernel launch from an ncu capture
# of the 512 x 512 workload at the benchmark's own 64 frames per launch
# (other frame counts are scaled by the frames).  Valid only for the kernel
# source the capture was taken on: any other source reports null.
TRAFFIC_CAPTURE = {"sources_sha256": "40a5c23cc3937400bd97127166354da7c89a78a0977c5891d9d93e252c61b0cb",
                   "frames": 64, "bytes": 32054272 + 79573760}


def beamform_traffic(frames):
    import hashlib

    src = os.path.join(ROOT, "paper_2311_00482_gb300", "csrc", "bf_kernels.cu")
    try:
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    if digest != TRAFFIC_CAPTURE["sources_sha256"]:
        return None
    return TRAFFIC_CAPTURE["bytes"] * frames / TRAFFIC_CAPTURE["frames"]


def max_over_ranks(x, device):
    """Largest x over the ranks of the default process group (x itself alone)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world_size, units_per_step, steps, seconds):
    """Whole-job throughput in giga-units/s: every rank does units_per_step per step
    (weak scaling), the job takes the slowest rank's time."""
    return world_size * units_per_step * steps / seconds / 1e9


def frames_rf(n_distinct=4):
    acq = synth.CYST_WIRES_512
    return acq, [synth.cyst_wires_frame(acq, seed=synth.BASE_SEED + 1 + k)[0] for k in range(n_distinct)]


def grid_of(acq):
    return (acq.nx, acq.nz, acq.x0_m, acq.x1_m, acq.z0_m, acq.z1_m)


def nominal_units(acq):
    return acq.nx * acq.nz * acq.n_elements * len(acq.angles_deg)


# ------------------------------------------------------------------ CPU --

def time_oracle(acq, rfs, budget_s, max_frames=2000):
    """FP64 oracle (beamform + envelope + log for DAS and DMAS) on host cores."""
    import oracle

    grid = grid_of(acq)
    dz = (acq.z1_m - acq.z0_m) / (acq.nz - 1)

    def one(rf):
        r = oracle.beamform(rf, acq.x_elements(), acq.angles_rad, grid, acq.fs_hz, acq.c_mps,
                            acq.f_number)
        oracle.log_compress(oracle.envelope(r["das"]))
        oracle.log_compress(oracle.envelope(r["dmas"], bandpass=True, dz=dz, c=acq.c_mps,
                                            f0=acq.f0_hz))

    t0 = time.perf_counter()
    one(rfs[0])
    t1 = time.perf_counter() - t0
    n = int(max(1, min(max_frames, budget_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    for k in range(n):
        one(rfs[k % len(rfs)])
    dt = time.perf_counter() - t0
    return dict(value=n * nominal_units(acq) / dt / 1e9, unit=UNIT, cores=oracle.max_threads(),
                kind="oracle", frames=n, seconds=dt,
                sample="%d frames of the 512x512 workload (DAS+DMAS, envelope, log), FP64, "
                       "OpenMP over pixels" % n)


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    acq, rfs = frames_rf(2)
    import oracle

    grid = grid_of(acq)
    dz = (acq.z1_m - acq.z0_m) / (acq.nz - 1)

    def step(rf):
        r = oracle.beamform(rf, acq.x_elements(), acq.angles_rad, grid, acq.fs_hz, acq.c_mps,
                            acq.f_number)
        oracle.log_compress(oracle.envelope(r["das"]))
        oracle.log_compress(oracle.envelope(r["dmas"], bandpass=True, dz=dz, c=acq.c_mps,
                                            f0=acq.f0_hz))

    for k in range(args.warmup):
        step(rfs[k % 2])
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        step(rfs[k % 2])
        times.append(time.perf_counter() - t0)
    t = sum(times)
    value = args.steps * nominal_units(acq) / t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "frames_per_s": args.steps / t,
        "config": {"workload": WORKLOAD, "frames_per_step": 1,
                   "note": "FP64 CPU oracle; each step is one frame (bounded sample)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(),
                         "kind": "oracle", "sample": "1 frame per step, %d steps" % args.steps},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU --

class ClockSampler:
    QUERY = ("clocks.sm,clocks.max.sm,utilization.gpu,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        rows = []
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), float(parts[2]), parts[4:8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        busy = [r for r in rows if r[2] >= 50] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in busy for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in busy), "sm_max_mhz": rows[0][1],
                "reasons": reasons, "samples": len(busy)}


def run_ours(args):
    import torch

    ws, rank, local = dist_info()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2311_00482_gb300 import build as bfbuild

    bfbuild.build()
    import paper_2311_00482_gb300 as bf

    bf.load()
    prec = {"fp32": bf.BF_PREC_FP32, "fp16": bf.BF_PREC_FP16, "bf16": bf.BF_PREC_BF16}[args.prec]
    flags = bf.BF_DAS | bf.BF_DMAS | bf.BF_OUT_LOGDB | prec
    acq, rfs = frames_rf(4)
    B = args.frames
    grid = grid_of(acq)
    h = bf.bf_create(acq.n_elements, acq.pitch_m, acq.f_number, grid, acq.fs_hz, acq.f0_hz,
                     acq.c_mps)
    # active (pixel, channel, angle) triples: the beamformer's algorithmic work
    valid, _ = bf.bf_host_tables(acq.n_elements, acq.pitch_m, acq.f_number, grid, acq.fs_hz,
                                 acq.f0_hz, acq.c_mps, acq.n_samples, acq.angles_rad)
    active = int(np.clip(valid[..., 1] - valid[..., 0] + 1, 0, None).sum())
    nm = 2
    # tile configuration from the library's autotuner (setup, not timed)
    if args.no_tune:
        tune = {"rows": bf.bf_plan_info(h, acq.n_samples, acq.angles_rad, flags)["rows"],
                "stage_bytes": None, "candidates_us": None}
    else:
        tune = bf.bf_autotune(h, acq.n_samples, acq.angles_rad, flags, frames=min(B, 16))
    rf_dev = [torch.from_numpy(rfs[k % len(rfs)]).to(dev) for k in range(B)]
    out_dev = [torch.empty((nm, acq.nx, acq.nz), dtype=torch.float32, device=dev) for _ in range(B)]
    batch = bf.Batch([(h, rf_dev[k], acq.n_samples, acq.angles_rad, flags, out_dev[k])
                      for k in range(B)])
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def barrier():
        if ws > 1:
            import torch.distributed as dist

            dist.barrier()

    # ---- device leg
    sampler = ClockSampler(local)
    sampler.start()
    for _ in range(args.warmup):
        flush.fill_(1)
        batch.launch(stream)
    torch.cuda.synchronize(dev)
    batch.status(stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize(dev)
    split = []
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        batch.launch(stream)
        ev[k][1].record(stream)
        # the per-kernel marks are events captured in the graph: read them after
        # each step (the wait sits outside the step's own event pair)
        ev[k][1].synchronize()
        split.append(batch.timing()[0])
    torch.cuda.synchronize(dev)
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    _, launches = batch.timing()
    ingest_ms, beam_ms, post_ms = (statistics.median(x[i] for x in split) for i in range(3))
    bf_ms = [x[1] for x in split]
    batch.status(stream)
    t_dev = max_over_ranks(sum(step_ms) / 1e3, dev)

    # ---- end-to-end leg through bf_submit / bf_poll (pinned host RF, host outputs)
    host_rf = [torch.from_numpy(rfs[k % len(rfs)]).pin_memory() for k in range(B)]
    # E2E_DEPTH steps in flight: step k + E2E_DEPTH is submitted before step k is
    # collected, so one set of host results per step in flight plus one
    # (each set one pinned buffer: the frames' images contiguous, so that a
    # batch's results leave in one transfer)
    host_out = [list(torch.empty((B, nm, acq.nx, acq.nz), dtype=torch.float32).pin_memory())
                for _ in range(E2E_DEPTH + 1)]
    # steps of the end-to-end leg: enough that filling and draining the
    # E2E_DEPTH steps in flight does not dominate (about 50 ms at 64 frames)
    e2e_steps = 50
    lat = []

    def e2e_run(steps, record):
        # each step's frames in one submission with their host destinations
        # (bf_submit_many_into: every RF copied on return; the batch delivers its
        # images to the pinned host buffers itself) and one collection
        # (bf_poll_many: waits for them); E2E_DEPTH steps stay in flight, so the
        # host->device copies, the kernels and the device->host copies of
        # different steps overlap.  A frame's latency: its step's submission to
        # every result of the step on the host.
        inflight = []
        for k in range(steps + E2E_DEPTH):
            if k < steps:
                t_sub = time.perf_counter()
                inflight.append((bf.bf_submit_many_into(h, host_rf, acq.n_samples, acq.angles_rad,
                                                        flags | bf.BF_DEST_ONE_BUFFER,
                                                        host_out[k % (E2E_DEPTH + 1)]),
                                 t_sub))
            if len(inflight) > E2E_DEPTH or (k >= steps and inflight):
                tickets, t_sub0 = inflight.pop(0)
                assert bf.bf_poll_many(h, tickets, None, timeout_us=30_000_000) == bf.BF_OK
                if record:
                    lat.extend([time.perf_counter() - t_sub0] * B)

    if not args.no_e2e:
        e2e_run(max(2, args.warmup), False)
        barrier()
        t0 = time.perf_counter()
        e2e_run(e2e_steps, True)
        t_e2e = time.perf_counter() - t0
    clocks = sampler.stop()
    if not args.no_e2e:
        t_e2e = max_over_ranks(t_e2e, dev)

    # ---- results (rank 0)
    units_step = B * nominal_units(acq)
    value = job_value(ws, units_step, args.steps, t_dev)
    props = torch.cuda.get_device_properties(dev)
    sm_count = props.multi_processor_count
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    sm_max = 2070.0
    if os.path.exists(peaks_path):
        try:
            sm_max = float(json.load(open(peaks_path)).get("sm_max_mhz", sm_max))
        except (OSError, ValueError):
            pass
    # Binding unit of DAS+DMAS: the special-function units (16 per SM per
    # clock).  Each frame's active triple needs its own signed square root
    # (DMAS); the receive distance's square root belongs to the (pixel,
    # channel, angle) geometry, which the step's B frames share, so it costs
    # at least 1 / B per frame's triple.
    sfu_per_triple = 1.0 + 1.0 / B
    peak_pch = sm_count * 16 * sm_max * 1e6 / sfu_per_triple
    beam_s = statistics.median(bf_ms) / 1e3 if bf_ms else beam_ms / 1e3
    achieved_pch = B * active / beam_s
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp16": "f16-storage/f32", "bf16": "bf16-storage/f32"}[args.prec],
        "data": "synthetic",
        "frames_per_s": ws * B * args.steps / t_dev,
        "latency_ms": None if args.no_e2e else {
            "p50": 1e3 * float(np.percentile(lat, 50)),
            "p99": 1e3 * float(np.percentile(lat, 99)),
            "source": "e2e leg: a step's %d frames submitted together (%d steps in flight), "
                      "latency from submission to every result of the step on the host"
                      % (B, E2E_DEPTH)},
        "config": {"workload": WORKLOAD, "frames_per_step": B, "global_batch": B * ws,
                   "parallelism": "replicas (frames sharded, no collective)",
                   "l2": "flushed before every timed step (256 MiB write)",
                   "active_triples_per_frame": active,
                   "precision": args.prec,
                   "tile": {"rows_per_thread": tune["rows"], "stage_bytes": tune["stage_bytes"],
                            "autotune_candidates_us": tune["candidates_us"]}},
        "kernel_ms": {"ingest": ingest_ms, "beamform": beam_ms, "envelope_log": post_ms},
        "roofline": {"bound": "alu", "kernel": "beamform_kernel",
                     "achieved": achieved_pch / 1e9, "peak": peak_pch / 1e9,
                     "unit": "G active pixel*ch/s", "frac": achieved_pch / peak_pch,
                     "peak_basis": "%d SMs x 16 SFU/clk x %.0f MHz / (1 signed root per frame's "
                                   "triple + 1 receive-distance root per (pixel, channel, angle) "
                                   "shared by the step's %d frames)" % (sm_count, sm_max, B),
                     "traffic": beamform_traffic(B),
                     "traffic_unit": "DRAM bytes per launch (ncu capture at 64 frames per launch)"},
        "e2e": None if args.no_e2e else {
            "value": job_value(ws, units_step, e2e_steps, t_e2e), "unit": UNIT,
            "h2d_bytes_per_step": B * rfs[0].nbytes,
            "d2h_bytes_per_step": B * nm * acq.nx * acq.nz * 4,
            "frames_per_s": ws * B * e2e_steps / t_e2e},
        "gpu_launches": launches * args.steps,
        "clocks": clocks,
    }
    if rank == 0 and not args.no_serving:
        # serving latency beside throughput: a short Poisson-served leg (not part
        # of the timed steps above)
        line["serving_latency_ms"] = serving_latency(torch, bf)
    if rank == 0 and ws == 1 and not args.no_cpu:
        line["cpu_baseline"] = time_oracle(acq, rfs, args.cpu_seconds)
    batch.close()
    bf.bf_destroy(h)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


# ----------------------------------------------------- informational modes --

def _setup_gpu():
    import torch

    from paper_2311_00482_gb300 import build as bfbuild

    bfbuild.build()
    import paper_2311_00482_gb300 as bf

    bf.load()
    torch.cuda.set_device(0)
    return torch, bf


def _handle(bf, acq):
    return bf.bf_create(acq.n_elements, acq.pitch_m, acq.f_number, grid_of(acq), acq.fs_hz,
                        acq.f0_hz, acq.c_mps)


def run_batch256(args):
    """Uneven 256-frame batch (64..1024 pixels per side, 1..11 angles) in one graph."""
    torch, bf = _setup_gpu()
    specs = synth.mixed_batch_specs(256)
    base = synth.cyst_wires_frame(synth.CYST_WIRES_512)[0][0]  # 0 deg record, reused per angle
    frames, handles, keep, units, active = [], [], [], 0, 0
    for k, sp in enumerate(specs):
        na = sp["n_angles"]
        acq = synth.CYST_WIRES_512.with_(nx=sp["nx"], nz=sp["nz"], angles_deg=synth.angles_linspace(na))
        h = _handle(bf, acq)
        handles.append(h)
        rf = torch.from_numpy(np.broadcast_to(base, (na,) + base.shape).copy()).cuda()
        flags = (bf.BF_DAS if k % 2 == 0 else bf.BF_DMAS) | bf.BF_OUT_LOGDB
        out = torch.empty((1, acq.nx, acq.nz), dtype=torch.float32, device="cuda")
        keep += [rf, out]
        frames.append((h, rf, acq.n_samples, acq.angles_rad, flags, out))
        units += nominal_units(acq)
    batch = bf.Batch(frames)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    for _ in range(args.warmup):
        batch.launch(st)
    torch.cuda.synchronize()
    times, beam = [], []
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        batch.launch(st)
        b.record(st)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
        beam.append(batch.timing()[0][1])
    batch.status(st)
    t = statistics.median(times) / 1e3
    print(json.dumps({"workload": "uneven batch: 256 frames, 64..1024 px per side, 1..11 plane waves, "
                                  "64 ch x 2048 samples, DAS or DMAS, envelope + log, one CUDA graph",
                      "frames_per_s": 256 / t, "gpixel_ch_per_s": units / t / 1e9,
                      "ms_per_batch": 1e3 * t, "beamform_ms": statistics.median(beam),
                      "note": "0 deg cyst record reused for every angle (work is data-independent)"}),
          flush=True)
    batch.close()
    for h in handles:
        bf.bf_destroy(h)


def run_iq(args):
    """IQ-DAS + BB-DMAS (Eq. (4)) of the 512x512 workload, 64 frames in one graph,
    log-compressed magnitude images; rel-L2 of one frame against the oracle."""
    import oracle

    torch, bf = _setup_gpu()
    acq, rfs = frames_rf(4)
    B = args.frames
    h = _handle(bf, acq)
    flags = bf.BF_IQDAS | bf.BF_BBDMAS | bf.BF_OUT_LOGDB
    if args.no_tune:
        tune = {"rows": bf.bf_plan_info(h, acq.n_samples, acq.angles_rad, flags)["rows"]}
    else:
        tune = bf.bf_autotune(h, acq.n_samples, acq.angles_rad, flags, frames=16)
    rf_dev = [torch.from_numpy(rfs[k % len(rfs)]).cuda() for k in range(B)]
    out_dev = [torch.empty((2, acq.nx, acq.nz), dtype=torch.float32, device="cuda") for _ in range(B)]
    batch = bf.Batch([(h, rf_dev[k], acq.n_samples, acq.angles_rad, flags, out_dev[k])
                      for k in range(B)])
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    for _ in range(args.warmup):
        batch.launch(st)
    torch.cuda.synchronize()
    times, split = [], []
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        batch.launch(st)
        b.record(st)
        b.synchronize()
        times.append(a.elapsed_time(b))
        split.append(batch.timing()[0])
    batch.status(st)
    t = sum(times) / 1e3
    # accuracy of the beamformed magnitudes on sampled pixels of one frame
    out = torch.empty((2, acq.nx, acq.nz), dtype=torch.float32, device="cuda")
    bf.bf_beamform(h, rf_dev[0], acq.n_samples, acq.angles_rad, bf.BF_IQDAS | bf.BF_BBDMAS, out)
    bf.bf_sync(h)
    pix = np.random.default_rng(3).integers(0, acq.nx * acq.nz, 20000)
    iq = oracle.demodulate(rfs[0], acq.fs_hz, acq.f0_hz)
    ref = oracle.beamform_iq(iq, acq.x_elements(), acq.angles_rad, grid_of(acq), acq.fs_hz,
                             acq.c_mps, acq.f_number, acq.f0_hz, pixels=pix)
    got = out.cpu().numpy().reshape(2, -1)[:, pix].astype(np.float64)
    err = {name: float(np.linalg.norm(got[k] - ref[name]) / np.linalg.norm(ref[name]))
           for k, name in enumerate(("iqdas", "bbdmas"))}
    batch.close()
    bf.bf_destroy(h)
    print(json.dumps({"workload": "IQ-DAS + BB-DMAS, cyst+wires 512x512 px, 64 ch, 2048 samples, 0 deg, "
                                  "demodulation + beamforming + log, %d frames per graph" % B,
                      "gpixel_ch_per_s": args.steps * B * nominal_units(acq) / t / 1e9,
                      "frames_per_s": args.steps * B / t, "ms_per_step": 1e3 * t / args.steps,
                      "kernel_ms": {"demod": statistics.median(x[0] for x in split),
                                    "beamform": statistics.median(x[1] for x in split),
                                    "log": statistics.median(x[2] for x in split)},
                      "tile": tune, "rel_l2": err,
                      "rel_l2_sample": "20000 random pixels of one frame vs the FP64 oracle"}),
          flush=True)


def run_fk(args):
    """Plane-wave f-k migration of the 64-channel, 2048-sample cyst record (one
    and three angles; the exact plane-wave mapping and Stolt's): time per frame
    on the device and rel-L2 against the oracle."""
    import oracle

    torch, bf = _setup_gpu()
    rows = []
    for angles in ((0.0,), (-7.0, 0.0, 7.0)):
        for mapping, flag, ref_fn in (("exact", 0, oracle.fk_migrate),
                                      ("stolt", bf.BF_FK_STOLT, oracle.fk_stolt)):
            acq = synth.CYST_WIRES_512.with_(angles_deg=angles)
            rf, _ = synth.cyst_wires_frame(acq)
            h = _handle(bf, acq)
            stream = torch.cuda.Stream()
            bf.bf_set_stream(h, stream)
            rf_d = torch.from_numpy(rf).cuda()
            out = torch.empty((acq.n_elements, acq.n_samples), dtype=torch.float32, device="cuda")
            for _ in range(5):
                bf.bf_fkmig(h, rf_d, acq.n_samples, acq.angles_rad, bf.BF_OUT_LOGDB | flag, out)
            torch.cuda.synchronize()
            ts = []
            for _ in range(50):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                bf.bf_fkmig(h, rf_d, acq.n_samples, acq.angles_rad, bf.BF_OUT_LOGDB | flag, out)
                b.record(stream)
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            bf.bf_fkmig(h, rf_d, acq.n_samples, acq.angles_rad, bf.BF_OUT_RF | flag, out)
            torch.cuda.synchronize()
            ref = ref_fn(rf, acq.pitch_m, acq.angles_rad, acq.fs_hz, acq.c_mps)
            got = out.cpu().numpy().astype(np.float64)
            err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
            t0 = time.perf_counter()
            ref_fn(rf, acq.pitch_m, acq.angles_rad, acq.fs_hz, acq.c_mps)
            cpu_ms = 1e3 * (time.perf_counter() - t0)
            rows.append({"mapping": mapping, "angles": len(angles), "gpu_ms": statistics.median(ts),
                         "frames_per_s": 1e3 / statistics.median(ts), "oracle_ms_numpy": cpu_ms,
                         "rel_l2": err})
            bf.bf_destroy(h)
    print(json.dumps({"workload": "plane-wave f-k migration, 64 ch x 2048 samples (cyst + wires), "
                                  "native grid 64 x 2048, -70 dB log, one frame per call",
                      "rows": rows}), flush=True)


def run_precision(args):
    """1024x1024, 128 elements, 4096 samples, 7 angles: time per frame and rel-L2 per storage."""
    import oracle

    torch, bf = _setup_gpu()
    acq = synth.PRECISION_1024
    rf, _ = synth.precision_frame(acq)
    h = _handle(bf, acq)
    rng = np.random.default_rng(5)
    pix = rng.integers(0, acq.nx * acq.nz, 20000)
    ref = oracle.beamform(rf, acq.x_elements(), acq.angles_rad, grid_of(acq), acq.fs_hz, acq.c_mps,
                          acq.f_number, pixels=pix)
    rf_d = torch.from_numpy(rf).cuda()
    stream = torch.cuda.Stream()  # the handle's work and the events below share it
    bf.bf_set_stream(h, stream)
    res = {}
    for name, prec in (("fp32", bf.BF_PREC_FP32), ("fp16", bf.BF_PREC_FP16), ("bf16", bf.BF_PREC_BF16)):
        flags = bf.BF_DAS | bf.BF_DMAS | bf.BF_CF | prec
        out = torch.empty((3, acq.nx, acq.nz), dtype=torch.float32, device="cuda")
        for _ in range(3):
            bf.bf_beamform(h, rf_d, acq.n_samples, acq.angles_rad, flags, out)
        bf.bf_sync(h)
        ts = []
        for _ in range(10):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            bf.bf_beamform(h, rf_d, acq.n_samples, acq.angles_rad, flags, out)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        got = out.cpu().numpy().reshape(3, -1)[:, pix].astype(np.float64)
        errs = {m: float(np.linalg.norm(got[k] - ref[m]) / np.linalg.norm(ref[m]))
                for k, m in enumerate(("das", "dmas", "cf"))}
        res[name] = {"ms_per_frame": statistics.median(ts), "rel_l2": errs,
                     "gpixel_ch_per_s": nominal_units(acq) / (statistics.median(ts) / 1e3) / 1e9}
    bf.bf_destroy(h)
    print(json.dumps({"workload": "1024x1024 px, 128 elements, 4096 samples, 7 plane waves over "
                                  "+-10 deg, DAS + DMAS + CF, beamformed output (single frames)",
                      "results": res, "rel_l2_sample": "20000 random pixels vs the FP64 oracle"}),
          flush=True)


def run_sweep(args):
    """The paper's grid sizes (depth x lateral), 50 MHz, 7.5 MHz probe, 3 cm, RF-DAS."""
    import oracle

    torch, bf = _setup_gpu()
    rows = []
    for nz, nx in synth.PAPER_GRIDS:
        acq = synth.Acquisition(f0_hz=7.5e6, fs_hz=50e6, n_samples=2048, nx=nx, nz=nz,
                                x0_m=-9.45e-3, x1_m=9.45e-3, z0_m=1e-3, z1_m=30e-3)
        rng = np.random.default_rng(7)
        ph = synth.make_phantom(acq, rng, n_speckle=3000, points=np.array([[0.0, 15e-3]]))
        rf = synth.synth_rf(acq, ph, rng)
        h = _handle(bf, acq)
        stream = torch.cuda.Stream()  # the handle's work and the events below share it
        bf.bf_set_stream(h, stream)
        rf_d = torch.from_numpy(rf).cuda()
        out = torch.empty((1, nx, nz), dtype=torch.float32, device="cuda")
        flags = bf.BF_DAS | bf.BF_OUT_LOGDB
        for _ in range(5):
            bf.bf_beamform(h, rf_d, acq.n_samples, acq.angles_rad, flags, out)
        bf.bf_sync(h)
        ts = []
        for _ in range(100):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            bf.bf_beamform(h, rf_d, acq.n_samples, acq.angles_rad, flags, out)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        def oracle_ms(threads, runs):
            cts = []
            for _ in range(runs):
                t0 = time.perf_counter()
                r = oracle.beamform(rf, acq.x_elements(), acq.angles_rad, grid_of(acq), acq.fs_hz,
                                    acq.c_mps, acq.f_number, threads=threads)
                oracle.log_compress(oracle.envelope(r["das"]))
                cts.append(1e3 * (time.perf_counter() - t0))
            return statistics.median(cts)

        g, c, c1 = statistics.median(ts), oracle_ms(0, 100), oracle_ms(1, 5)
        rows.append({"grid": "%dx%d" % (nz, nx), "gpu_ms": g, "cpu_oracle_ms": c,
                     "cpu_oracle_1core_ms": c1, "speedup": c / g, "speedup_1core": c1 / g})
        bf.bf_destroy(h)
    import oracle as _o

    print(json.dumps({"workload": "grid sweep of Sec. II-D, RF-DAS + envelope + log, one frame per call, "
                                  "median of 100 (GPU, FP64 oracle on %d threads) / 5 (oracle on 1 core)" % _o.max_threads(),
                      "rows": rows}), flush=True)


SERVING_WORKLOAD = ("serving: Poisson arrivals, square grids 128..1024 px, 1..7 plane waves, DAS or "
                    "DMAS, 64 ch x 2048 samples, pinned host RF in, pinned host dB image out; "
                    "engine = continuous batching with FP16 storage, plain = FIFO of one-frame "
                    "FP32 launches")


class ServingTrace:
    """Poisson arrivals of mixed requests, pinned host RF in and host dB images
    out: the continuous-batching engine (FP16 storage) against a FIFO in front
    of the plain FP32 one-frame-per-launch kernel, on the same trace."""

    def __init__(self, torch, bf, n_requests, seed=synth.BASE_SEED + 4):
        self.torch, self.bf, self.N = torch, bf, n_requests
        self.rng = np.random.default_rng(seed)
        base = synth.cyst_wires_frame(synth.CYST_WIRES_512)[0][0]
        self.rf_host = torch.from_numpy(
            np.ascontiguousarray(np.broadcast_to(base, (7,) + base.shape))).pin_memory()
        self.handles = {}
        self.trace = []
        for _ in range(n_requests):
            n = 64 * int(self.rng.integers(2, 17))  # 128 .. 1024 pixels per side
            na = int(self.rng.integers(1, 8))
            mode = bf.BF_DAS if self.rng.random() < 0.5 else bf.BF_DMAS
            self.trace.append((n, na, mode, np.deg2rad(synth.angles_linspace(na))))
        self.outs = {n: torch.empty((1, n, n), dtype=torch.float32).pin_memory()
                     for n, *_ in self.trace}
        self.stream = torch.cuda.Stream()
        self.rf_dev = torch.empty_like(self.rf_host, device="cuda")
        self.out_dev = torch.empty((1024 * 1024,), dtype=torch.float32, device="cuda")
        for h in set(self.handle(n) for n, *_ in self.trace):
            bf.bf_set_stream(h, self.stream)
        # untimed pass: every table, slot and scratch buffer exists before the clock starts
        seen = set()
        for k in range(self.N):
            if self.trace[k][:3] not in seen:
                seen.add(self.trace[k][:3])
                self.plain_run(k)
        for k0 in range(0, self.N, 128):  # in chunks: admission caps the requests in flight
            ks = range(k0, min(self.N, k0 + 128))
            tickets = [self.engine_submit(k) for k in ks]
            for k, t in zip(ks, tickets):
                self.engine_wait(k, t)

    def handle(self, n):
        if n not in self.handles:
            self.handles[n] = _handle(self.bf, synth.CYST_WIRES_512.with_(nx=n, nz=n))
        return self.handles[n]

    def engine_submit(self, k):
        bf = self.bf
        n, na, mode, ang = self.trace[k]
        while True:
            try:
                return bf.bf_submit(self.handle(n), self.rf_host[:na], 2048, ang,
                                    mode | bf.BF_PREC_FP16 | bf.BF_OUT_LOGDB)
            except bf.BFError as e:
                if e.code != bf.BF_EAGAIN:
                    raise

    def engine_wait(self, k, ticket):
        n = self.trace[k][0]
        self.bf.bf_poll(self.handle(n), ticket, self.outs[n], timeout_us=60_000_000)

    def plain_run(self, k):
        torch, bf = self.torch, self.bf
        n, na, mode, ang = self.trace[k]
        h = self.handle(n)
        nb = na * 64 * 2048
        with torch.cuda.stream(self.stream):
            self.rf_dev.view(-1)[:nb].copy_(self.rf_host.view(-1)[:nb], non_blocking=True)
            bf.bf_beamform_plain(h, self.rf_dev.view(-1)[:nb], 2048, ang, mode | bf.BF_OUT_LOGDB,
                                 self.out_dev[:n * n])
            self.outs[n].view(-1).copy_(self.out_dev[:n * n], non_blocking=True)
        self.stream.synchronize()

    def drive(self, rate, kind):
        """One pass of the trace at `rate` Hz; kind "batched_fp16" or "plain_fp32"."""
        import queue
        import threading

        N = self.N
        gaps = self.rng.exponential(1.0 / rate, N)
        lat, t_sub = [0.0] * N, [0.0] * N
        handoff = queue.Queue()

        def completer():
            for k in range(N):
                item = handoff.get()
                if kind == "batched_fp16":
                    self.engine_wait(k, item)
                else:
                    self.plain_run(k)
                lat[k] = time.perf_counter() - t_sub[k]

        th = threading.Thread(target=completer)
        th.start()
        t0 = time.perf_counter()
        t_next = t0
        for k in range(N):
            t_next += gaps[k]
            while time.perf_counter() < t_next:
                pass
            t_sub[k] = time.perf_counter()
            handoff.put(self.engine_submit(k) if kind == "batched_fp16" else k)
        th.join()
        t_all = time.perf_counter() - t0
        units = sum(n * n * 64 * na for n, na, _, _ in self.trace)
        return {"rate_hz": rate, "engine": kind, "frames_per_s": N / t_all,
                "gpixel_ch_per_s": units / t_all / 1e9,
                "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99))}

    def close(self):
        for h in self.handles.values():
            self.bf.bf_destroy(h)
        self.handles = {}


def serving_latency(torch, bf, n_requests=300, rates=(2000, 10000)):
    """The short serving leg of the default line: per rate the engine's and the
    plain kernel's frame latency (submission to the dB image on the host)."""
    sys.setswitchinterval(1e-5)  # the submitting thread spins; let the completion thread in
    st = ServingTrace(torch, bf, n_requests)
    try:
        rows = []
        for rate in rates:
            e = st.drive(rate, "batched_fp16")
            p = st.drive(rate, "plain_fp32")
            rows.append({"rate_hz": rate, "p50": e["p50_ms"], "p99": e["p99_ms"],
                         "frames_per_s": e["frames_per_s"], "plain_p50": p["p50_ms"],
                         "plain_p99": p["p99_ms"], "plain_frames_per_s": p["frames_per_s"]})
        return {"workload": SERVING_WORKLOAD, "requests_per_rate": n_requests, "rates": rows}
    finally:
        st.close()


def run_serving(args):
    """Poisson arrivals at 1, 2, 5, 10 and 20 kHz (see ServingTrace)."""
    torch, bf = _setup_gpu()
    sys.setswitchinterval(1e-5)  # the submitting thread spins; let the completion thread in
    st = ServingTrace(torch, bf, args.requests)
    results = []
    for rate in (1000, 2000, 5000, 10000, 20000):
        for kind in ("batched_fp16", "plain_fp32"):
            results.append(st.drive(rate, kind))
            print(json.dumps(results[-1]), flush=True)
    print(json.dumps({"workload": SERVING_WORKLOAD, "requests_per_rate": args.requests,
                      "results": results}), flush=True)
    st.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch256":
        run_batch256(args)
    elif args.workload == "precision":
        run_precision(args)
    elif args.workload == "iq":
        run_iq(args)
    elif args.workload == "fk":
        run_fk(args)
    elif args.workload == "sweep":
        run_sweep(args)
    elif args.workload == "serving":
        run_serving(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
