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
    return p.parse_args()


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def frames_rf(n_distinct=4):
    acq = synth.CYST_WIRES_512
    return acq, [synth.cyst_wires_frame(acq, seed=synth.BASE_SEED + 1 + k)[0] for k in range(n_distinct)]


def grid_of(acq):
    return (acq.nx, acq.nz, acq.x0_m, acq.x1_m, acq.z0_m, acq.z1_m)


def nominal_units(acq):
    return acq.nx * acq.nz * acq.n_elements * len(acq.angles_deg)


# ------------------------------------------------------------------ CPU --

def time_oracle(acq, rfs, budget_s, max_frames=64):
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
    bf_ms = []
    barrier()
    torch.cuda.synchronize(dev)
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        batch.launch(stream)
        ev[k][1].record(stream)
        if k == 0 or k == args.steps - 1:
            pass
    torch.cuda.synchronize(dev)
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    # per-kernel split of the last replay (events captured inside the graph)
    (ingest_ms, beam_ms, post_ms), launches = batch.timing()
    # the beamforming kernel over every timed step: replay once more per step with timing reads
    for k in range(min(args.steps, 10)):
        flush.fill_(3)
        batch.launch(stream)
        torch.cuda.synchronize(dev)
        bf_ms.append(batch.timing()[0][1])
    batch.status(stream)
    t_dev = sum(step_ms) / 1e3
    if ws > 1:
        import torch.distributed as dist

        t = torch.tensor([t_dev], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_dev = float(t.item())

    # ---- end-to-end leg through bf_submit / bf_poll (pinned host RF, host outputs)
    host_rf = [torch.from_numpy(rfs[k % len(rfs)]).pin_memory() for k in range(B)]
    host_out = [torch.empty((nm, acq.nx, acq.nz), dtype=torch.float32).pin_memory() for _ in range(B)]
    e2e_steps = max(2, min(args.steps, 10))
    lat = []

    def e2e_step(record):
        t_sub = []
        tickets = []
        for k in range(B):
            t_sub.append(time.perf_counter())
            tickets.append(bf.bf_submit(h, host_rf[k], acq.n_samples, acq.angles_rad, flags))
        for k in range(B):
            assert bf.bf_poll(h, tickets[k], host_out[k], timeout_us=30_000_000) == bf.BF_OK
            if record:
                lat.append(time.perf_counter() - t_sub[k])

    for _ in range(max(2, args.warmup)):
        e2e_step(False)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step(True)
    t_e2e = time.perf_counter() - t0
    clocks = sampler.stop()
    if ws > 1:
        import torch.distributed as dist

        t = torch.tensor([t_e2e], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_e2e = float(t.item())

    # ---- results (rank 0)
    units_step = B * nominal_units(acq)
    value = ws * units_step * args.steps / t_dev / 1e9
    props = torch.cuda.get_device_properties(dev)
    sm_count = props.multi_processor_count
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    sm_max = 2070.0
    if os.path.exists(peaks_path):
        try:
            sm_max = float(json.load(open(peaks_path)).get("sm_max_mhz", sm_max))
        except (OSError, ValueError):
            pass
    # Binding unit of DAS+DMAS: two square roots per active triple on the
    # special-function units (16 per SM per clock).
    peak_pch = sm_count * 16 * sm_max * 1e6 / 2.0
    beam_s = statistics.median(bf_ms) / 1e3 if bf_ms else beam_ms / 1e3
    achieved_pch = B * active / beam_s
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp16": "f16-storage/f32", "bf16": "bf16-storage/f32"}[args.prec],
        "data": "synthetic",
        "frames_per_s": ws * B * args.steps / t_dev,
        "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)),
                       "p99": 1e3 * float(np.percentile(lat, 99)),
                       "source": "e2e leg, submit -> result on host, %d frames in flight" % B},
        "config": {"workload": WORKLOAD, "frames_per_step": B, "global_batch": B * ws,
                   "parallelism": "replicas (frames sharded, no collective)",
                   "l2": "flushed before every timed step (256 MiB write)",
                   "active_triples_per_frame": active,
                   "precision": args.prec},
        "kernel_ms": {"ingest": ingest_ms, "beamform": beam_ms, "envelope_log": post_ms},
        "roofline": {"bound": "alu", "kernel": "beamform_kernel",
                     "achieved": achieved_pch / 1e9, "peak": peak_pch / 1e9,
                     "unit": "G active pixel*ch/s", "frac": achieved_pch / peak_pch,
                     "peak_basis": "%d SMs x 16 SFU/clk x %.0f MHz / 2 square roots per triple"
                                   % (sm_count, sm_max),
                     "traffic": None},
        "e2e": {"value": ws * units_step * e2e_steps / t_e2e / 1e9, "unit": UNIT,
                "h2d_bytes_per_step": B * rfs[0].nbytes,
                "d2h_bytes_per_step": B * nm * acq.nx * acq.nz * 4,
                "frames_per_s": ws * B * e2e_steps / t_e2e},
        "gpu_launches": launches * args.steps,
        "clocks": clocks,
    }
    if rank == 0 and ws == 1 and not args.no_cpu:
        line["cpu_baseline"] = time_oracle(acq, rfs, args.cpu_seconds)
    batch.close()
    bf.bf_destroy(h)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
