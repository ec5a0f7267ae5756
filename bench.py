"""Benchmark: RAAR frame-iterations/s on one GB300 for the 2500-frame 128^2
Fermat-spiral scan over a 1024^2 object (probe refinement every 2nd step,
eps_a every step, eps_Q and eps_Delta every 10th), with the fused frame kernel's HBM roofline fraction,
an end-to-end figure through the C ABI with host buffers, and the FP64 oracle
timed on the host cores as a reported CPU baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload fermat|raster256|batch|batch-small] [--no-mixed]
                  [--copy-streams S]

--workload raster256 times the large scan instead: a 100 x 100 raster of
256^2 frames (step 24 +-1 px) over a 3072^2 object, Poisson 10^8 photons,
fixed probe.

For 128^2 workloads the line also carries "mixed": the same steps with the
frame DFTs as FP16 (per-frame scaled) and BF16x3 tensor-core contractions,
each with its frame-kernel time, HBM fraction and tensor rate.

Prints one JSON line on rank 0.  Under torchrun (N > 1) every rank runs an
independent replica of the scan (the path has no exchange step on one box),
so scaling is weak and value = all ranks' frame-iterations / slowest rank.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RAAR frame-iterations/s on 1 GB300 (FP32 vs mixed) and % of HBM roofline"
UNIT = "frame-iterations/s"
WORKLOAD = "fermat-2500x128-obj1024"
RESIDUAL_EVERY = 10   # eps_Q and eps_Delta every 10th step; eps_a every step
PROFILES = {"fermat": os.path.join(ROOT, "profiles", "raar_kernel_fermat128.txt"),
            "raster256": os.path.join(ROOT, "profiles", "big_kernel_raster256.txt")}
CSRC = os.path.join(ROOT, "paper_1602_01448_gb300", "csrc")


# Sources that make up each workload's frame-pass kernel: a committed ncu
# summary stays valid while these hash to the profiled version.
KERNEL_SOURCES = {
    "fermat": ["raar_kernel.cuh", "fft_frame.cuh", "tma.cuh", "sharp_common.cuh", "gen_twiddles.py",
               "raar_128_w0.cu"],
    "raster256": ["frame256.cuh", "frame256_raar.cu", "fft_frame.cuh", "tma.cuh", "sharp_common.cuh",
                  "gen_twiddles.py"],
}


def kernel_source_hash(workload: str = "fermat") -> str:
    h = hashlib.sha256()
    for name in sorted(KERNEL_SOURCES[workload]):
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str = "fermat"):
    """DRAM bytes per launch of the frame kernel from the committed ncu
    summary, or None when the kernel sources changed since it was taken."""
    try:
        text = open(PROFILES[workload]).read()
    except OSError:
        return None
    mh = re.search(r"source_hash:\s*([0-9a-f]+)", text)
    mt = re.search(r"dram_bytes_per_launch_full:\s*([0-9.eE+]+)", text)
    if not mh or not mt or mh.group(1) != kernel_source_hash(workload):
        return None
    return float(mt.group(1))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def measured_peak_tensor():
    """Measured dense BF16 tensor rate (TFLOP/s, burst) of this machine's GPUs;
    FP16 has the same nominal dense rate."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1900.0


def slowest_rank_ms(ms: float, world: int, device=None) -> float:
    """Max over ranks of a per-rank time (the job is as slow as its slowest
    replica); identity for a single process."""
    if world <= 1:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(frames_per_rank: int, steps: int, world: int, ms_total: float) -> float:
    """Whole-job frame-iterations per second: every rank runs its own replica
    of the scan (weak scaling), timed by the slowest rank."""
    return world * frames_per_rank * steps / (ms_total / 1000.0)


def make_scan(frames=None, workload: str = "fermat"):
    import synth
    if workload == "raster256":
        side = 100 if frames is None else max(1, int(round(math.sqrt(frames))))
        return synth.scan_large_raster(side=side)
    return synth.scan_fermat(count=2500 if frames is None else frames)


def device_poisson(amp, photons: float, seed: int):
    """Poisson-noisy amplitudes drawn on the device (same recipe as
    synth.poisson_intensities: every frame scaled to `photons` counts in
    total), for workloads too large to draw on the host in reasonable time."""
    import torch
    g = torch.Generator(device=amp.device)
    g.manual_seed(seed)
    out = torch.empty_like(amp)
    for k0 in range(0, amp.shape[0], 1000):
        inten = amp[k0:k0 + 1000].double() ** 2
        tot = inten.sum(dim=(1, 2), keepdim=True)
        scale = torch.where(tot > 0, photons / tot.clamp_min(1e-300), torch.zeros_like(tot))
        counts = torch.poisson(inten * scale, generator=g)
        out[k0:k0 + 1000] = torch.where(scale > 0, counts / scale.clamp_min(1e-300),
                                        torch.zeros_like(counts)).sqrt().float()
    return out


def oracle_sample_rate(scan, amps, n_frames: int, n_steps: int = 1):
    """FP64 oracle RAAR steps over the first n_frames frames of the scan (full
    object): frame-iterations per second of host time."""
    import oracle as O
    pos = scan.pos[:n_frames]
    a = amps[:n_frames]
    z = O.split(scan.psi_init, scan.probe_init, pos)
    t0 = time.perf_counter()
    for _ in range(n_steps):
        z = O.raar_update(z, a, scan.probe_init, pos, scan.shape, 0.75)
        O.object_update(z, scan.probe_init, pos, scan.shape)
    dt = time.perf_counter() - t0
    return n_frames * n_steps / dt, dt


def host_amplitudes(scan, seed=5):
    """Noisy amplitudes for the oracle arms, computed with the oracle's forward
    model (the GPU arm computes its own with the library)."""
    import oracle as O
    import synth
    inten = O.forward_amplitudes(scan.obj, scan.probe, scan.pos) ** 2
    return np.sqrt(synth.poisson_intensities(inten, scan.photons, seed))


def run_reference(args, rank):
    if rank != 0:
        return
    scan = make_scan()
    n = 500
    import oracle as O
    import synth
    inten = O.forward_amplitudes(scan.obj, scan.probe, scan.pos[:n]) ** 2
    a = np.sqrt(synth.poisson_intensities(inten, scan.photons, 5))
    for _ in range(args.warmup):
        oracle_sample_rate(scan, a, n)
    times = []
    for _ in range(args.steps):
        _, dt = oracle_sample_rate(scan, a, n)
        times.append(dt)
    ms = 1000.0 * float(np.mean(times))
    val = n / (ms / 1000.0)
    sample = f"first {n} of 2500 frames per step, full 1024^2 object, FP64 NumPy"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def time_mixed(S, scan, amp, psi0, w0, prec, steps, warmup, world, dev):
    """The same RAAR steps with the frame DFTs as tensor-core contractions
    (precision `prec`, 128^2 frames): throughput, frame-kernel time, its HBM
    fraction (20 m^2 B per frame) and its tensor-pipe rate (4 complex
    128 x 128 x 128 products per frame = 16 real ones, 2 m^3 flops each; the
    BF16 three-term split issues each real product three times)."""
    import torch
    K, m = scan.K, scan.m
    plan = S.Plan(scan.pos, m, scan.shape, beta=0.75, probe_every=scan.probe_every,
                  residual_every=RESIDUAL_EVERY, device=dev, precision=prec)
    plan.raar_init(psi0, w0)
    for _ in range(warmup):
        plan.raar_step(amp)
    torch.cuda.synchronize()
    S.sharp_plan_set_profiling(plan.handle, True)
    S.sharp_plan_kernel_times(plan.handle)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        plan.raar_step(amp)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_total = slowest_rank_ms(e0.elapsed_time(e1), world, dev)
    kt = S.sharp_plan_kernel_times(plan.handle)
    S.sharp_plan_set_profiling(plan.handle, False)
    plan.status()
    frame_ms, frame_n = kt["frame"]
    t_frame = frame_ms / max(frame_n, 1) / 1000.0
    peak_hbm, _ = measured_peak_hbm()
    terms = 3 if prec == "bf16x3" else 1
    flops = 16 * 2.0 * m ** 3 * terms * K
    peak_tc = measured_peak_tensor()
    met = plan.metrics.cpu().numpy().tolist()
    launches = sum(n for _, n in kt.values())
    out = {"precision": prec, "value": job_throughput(K, steps, world, ms_total), "unit": UNIT,
           "ms_per_step": ms_total / steps, "frame_kernel_ms": t_frame * 1000.0,
           "hbm": {"achieved": 20.0 * m * m * K / t_frame / 1e9, "peak": peak_hbm, "unit": "GB/s",
                   "frac": 20.0 * m * m * K / t_frame / 1e9 / peak_hbm},
           "tensor": {"achieved": flops / t_frame / 1e12, "peak": peak_tc, "unit": "TFLOP/s",
                      "frac": flops / t_frame / 1e12 / peak_tc if peak_tc else None,
                      "flops_per_launch": flops, "terms": terms},
           "gpu_launches": launches, "last_metrics": {"eps_a": met[0], "eps_q": met[1]}}
    plan.close()
    return out


def run_ours(args, rank, world):
    import torch
    import paper_1602_01448_gb300 as S
    import synth

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    scan = make_scan(args.frames, args.workload)
    K, m = scan.K, scan.m
    plan = S.Plan(scan.pos, m, scan.shape, beta=0.75, probe_every=scan.probe_every, residual_every=RESIDUAL_EVERY,
                  device=dev)
    obj = torch.as_tensor(scan.obj).to(torch.complex64).to(dev)
    probe_true = torch.as_tensor(scan.probe).to(torch.complex64).to(dev)
    amp = plan.forward_amplitudes(obj, probe_true)
    if args.workload == "fermat":
        inten = (amp.double() ** 2).cpu().numpy()
        amp_h = np.sqrt(synth.poisson_intensities(inten, scan.photons, 5)).astype(np.float32)
        amp = torch.as_tensor(amp_h).to(dev)
    else:
        amp = device_poisson(amp, scan.photons, 5)
    psi0 = torch.as_tensor(scan.psi_init).to(torch.complex64).to(dev)
    w0 = torch.as_tensor(scan.probe_init).to(torch.complex64).to(dev)
    plan.raar_init(psi0, w0)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        plan.raar_step(amp)
    torch.cuda.synchronize()
    S.sharp_plan_set_profiling(plan.handle, True)
    S.sharp_plan_kernel_times(plan.handle)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.raar_step(amp)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms_total = e0.elapsed_time(e1)
    kt = S.sharp_plan_kernel_times(plan.handle)
    S.sharp_plan_set_profiling(plan.handle, False)
    metrics = plan.metrics.cpu().numpy().tolist()
    ms_total = slowest_rank_ms(ms_total, world, dev)
    ms_step = ms_total / args.steps
    value = job_throughput(K, args.steps, world, ms_total)

    # roofline of the fused frame kernel: 20 m^2 B per frame-iteration
    frame_ms, frame_n = kt["frame"]
    t_frame = frame_ms / max(frame_n, 1) / 1000.0
    alg_bytes = 20.0 * m * m * K
    achieved = alg_bytes / t_frame / 1e9
    peak, peak_kind = measured_peak_hbm()
    launches = sum(n for _, n in kt.values())

    # end to end through the C ABI with host buffers: every step uploads its
    # measured amplitudes from pinned host memory and reads the object back.
    # The upload for step k+1 runs on its own stream while step k computes
    # (two device buffers), and the object of step k is read back on a third
    # stream from a device snapshot; every copy of the timed steps lies
    # inside the timed region (the first upload starts after the start event,
    # the end event waits for the last read-back).
    e2e_steps = max(4, min(args.steps, 10))
    amp_pin = torch.empty(amp.shape, dtype=amp.dtype, pin_memory=True)
    amp_pin.copy_(amp)
    amp_dev = [torch.empty_like(amp), torch.empty_like(amp)]
    psi_snap = [torch.empty_like(plan.psi), torch.empty_like(plan.psi)]
    psi_pin = [torch.empty(plan.psi.shape, dtype=plan.psi.dtype, pin_memory=True) for _ in range(2)]
    # the upload of a step is split into contiguous slices, one copy stream
    # each, so that several copy engines share the host-to-device transfer
    n_up = max(1, args.copy_streams)
    up_s = [torch.cuda.Stream(device=dev) for _ in range(n_up)]
    down_s = torch.cuda.Stream(device=dev)
    flat_pin = amp_pin.view(-1)
    bounds = [(len(flat_pin) * j) // n_up for j in range(n_up + 1)]
    uploaded = [[torch.cuda.Event() for _ in range(n_up)] for _ in range(2)]
    consumed = [torch.cuda.Event(), torch.cuda.Event()]
    snapped = [torch.cuda.Event(), torch.cuda.Event()]
    read = [torch.cuda.Event(), torch.cuda.Event()]
    torch.cuda.synchronize()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)

    def upload(k):
        b = k % 2
        dst = amp_dev[b].view(-1)
        for j, st in enumerate(up_s):
            st.wait_event(f0)
            if k >= 2:
                st.wait_event(consumed[b])        # step k-2 is done with this buffer
            with torch.cuda.stream(st):
                dst[bounds[j]:bounds[j + 1]].copy_(flat_pin[bounds[j]:bounds[j + 1]], non_blocking=True)
            uploaded[b][j].record(st)

    upload(0)
    for k in range(e2e_steps):
        b = k % 2
        if k + 1 < e2e_steps:
            upload(k + 1)
        for ev in uploaded[b]:
            stream.wait_event(ev)
        if k >= 2:
            stream.wait_event(read[b])           # snapshot buffer b was read back
        plan.raar_step(amp_dev[b])
        consumed[b].record(stream)
        psi_snap[b].copy_(plan.psi)
        snapped[b].record(stream)
        down_s.wait_event(snapped[b])
        with torch.cuda.stream(down_s):
            psi_pin[b].copy_(psi_snap[b], non_blocking=True)
        read[b].record(down_s)
    stream.wait_event(read[(e2e_steps - 1) % 2])
    stream.wait_event(read[(e2e_steps - 2) % 2])
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = f0.elapsed_time(f1) / e2e_steps
    e2e_ms = slowest_rank_ms(e2e_ms, world, dev)

    mixed = []
    if m == 128 and not args.no_mixed:
        for prec in ("fp16s", "bf16x3"):
            mixed.append(time_mixed(S, scan, amp, psi0, w0, prec, args.steps, args.warmup, world, dev))

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        n = K if m <= 128 else 300
        import oracle as O
        inten = O.forward_amplitudes(scan.obj, scan.probe, scan.pos[:n]) ** 2
        a_o = np.sqrt(synth.poisson_intensities(inten, scan.photons, 5))
        rate, dt = oracle_sample_rate(scan, a_o, n, 1)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one FP64 RAAR step + object update over {n} of {K} frames "
                         f"(full {scan.shape[0]}^2 object), {dt:.1f} s, NumPy single thread"}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": scan.name, "frames": K, "frame": m, "object": list(scan.shape),
                   "beta": 0.75, "probe_every": scan.probe_every, "residual_every": RESIDUAL_EVERY,
                   "photons_per_frame": scan.photons, "parallelism": f"replicas{world}",
                   "l2": f"inputs larger than L2 (c {8 * K * m * m / 1e6:.0f} MB + a {4 * K * m * m / 1e6:.0f} MB per step)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": profiled_traffic(args.workload) if args.frames is None else None,
                     "kernel": "raar_kernel<128>" if m <= 128 else "big_kernel<RAAR> (256^2 line passes)",
                     "peak_kind": peak_kind,
                     "alg_bytes_per_launch": alg_bytes, "kernel_ms": t_frame * 1000.0},
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in kt.items()},
        "cpu_baseline": cpu,
        "e2e": {"value": world * K / (e2e_ms / 1000.0), "unit": UNIT,
                "h2d_bytes_per_step": int(amp.numel() * 4), "d2h_bytes_per_step": int(plan.psi.numel() * 8),
                "ms_per_step": e2e_ms, "copy_streams": n_up},
        "gpu_launches": launches,
        "clocks": clocks,
        "last_metrics": {"eps_a": metrics[0], "eps_q": metrics[1]},
        # the same workload with the frame DFTs as tensor-core contractions
        # (FP16 per-frame scaled; BF16 three-term), timed after the FP32 run
        "mixed": mixed,
    }
    print(json.dumps(out), flush=True)


def batch_scans(n_scans: int = 32, seed: int = 7, small: bool = False):
    """32 independent scans: frame size drawn from {64, 128, 256}, frame count
    uniform in [100, 4000]; each a raster of side ceil(sqrt(K)) with step
    round(0.1875 m), object = scan extent + 64 px, Poisson 10^U[5,7].
    small=True: 128 scans of 100 frames of 64^2 (many small scans, where the
    per-scan launches dominate)."""
    import synth
    if small:
        return [synth.scan_batch_member(300 + i, 64, 100) for i in range(128)]
    rng = np.random.default_rng(seed)
    ms = rng.choice([64, 128, 256], size=n_scans)
    ks = rng.integers(100, 4001, size=n_scans)
    return [synth.scan_batch_member(100 + i, int(m), int(k)) for i, (m, k) in enumerate(zip(ms, ks))]


def run_batch(args, rank, world):
    """Batched multi-scan RAAR: every step runs one persistent frame pass per
    frame size over all scans (sharp_batch_step, replayed as a CUDA graph);
    compared with stepping the same scans one after another."""
    import torch
    import paper_1602_01448_gb300 as S

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    scans = batch_scans(small=args.workload == "batch-small")
    total = sum(sc.K for sc in scans)
    alg_bytes = sum(20.0 * sc.m * sc.m * sc.K for sc in scans)

    def make(sc, amp=None):
        plan = S.Plan(sc.pos, sc.m, sc.shape, beta=0.75, residual_every=RESIDUAL_EVERY, device=dev)
        if amp is None:
            a = plan.forward_amplitudes(torch.as_tensor(sc.obj).to(torch.complex64).to(dev),
                                        torch.as_tensor(sc.probe).to(torch.complex64).to(dev))
            amp = device_poisson(a, sc.photons, sc.seed)
        plan.raar_init(torch.as_tensor(sc.psi_init).to(torch.complex64).to(dev),
                       torch.as_tensor(sc.probe_init).to(torch.complex64).to(dev))
        return plan, amp

    made = [make(sc) for sc in scans]
    plans, amps = [p for p, _ in made], [a for _, a in made]
    batch = S.Batch(plans, amps)
    stream = torch.cuda.current_stream()

    def timed(fn, steps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    for _ in range(max(args.warmup, 4)):        # includes the grid autotuning steps
        batch.step()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ms_total = timed(batch.step, args.steps)
    clocks = sampler.stop()
    batch.status()
    ms_total = slowest_rank_ms(ms_total, world, dev)
    ms_step = ms_total / args.steps

    # the same scans stepped one after another through sharp_raar_step
    singles = [make(sc, a)[0] for sc, a in zip(scans, amps)]

    def one_by_one():
        for p, a in zip(singles, amps):
            p.raar_step(a)

    for _ in range(args.warmup):
        one_by_one()
    ms_single = timed(one_by_one, args.steps) / args.steps
    if rank != 0:
        return
    grids = {m: batch.tuned_grid(m) for m in (64, 128, 256)}
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle as O
        import synth
        sc = scans[0]
        n = min(sc.K, 300)
        inten = O.forward_amplitudes(sc.obj, sc.probe, sc.pos[:n]) ** 2
        a_o = np.sqrt(synth.poisson_intensities(inten, sc.photons, 5))
        rate, dt = oracle_sample_rate(sc, a_o, n, 1)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one FP64 RAAR step + object update over {n} frames of {sc.m}^2 "
                         f"(first scan of the batch), {dt:.1f} s, NumPy single thread"}
    peak, peak_kind = measured_peak_hbm()
    achieved = alg_bytes / (ms_step / 1000.0) / 1e9
    out = {
        "metric": METRIC, "value": world * total * args.steps / (ms_total / 1000.0), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"batch-{len(scans)}scans-{total}frames", "scans": len(scans), "frames": total,
                   "frames_by_size": {str(m): sum(sc.K for sc in scans if sc.m == m) for m in (64, 128, 256)},
                   "beta": 0.75, "probe_every": 0, "residual_every": RESIDUAL_EVERY,
                   "parallelism": f"replicas{world}", "tuned_grid": grids,
                   "l2": f"inputs larger than L2 ({alg_bytes * 0.6 / 1e9:.1f} GB of state + amplitudes read per step)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "whole step (all launches of sharp_batch_step)",
                     "peak_kind": peak_kind, "alg_bytes_per_launch": alg_bytes, "kernel_ms": ms_step},
        "one_by_one": {"ms_per_step": ms_single, "value": total / (ms_single / 1000.0),
                       "speedup_of_batch": ms_single / ms_step},
        "cpu_baseline": cpu,
        "e2e": None,
        # per step: one frame pass per frame size, then per scan the image
        # pass and the metric finalisation (no probe updates in this workload)
        "gpu_launches": args.steps * (len({sc.m for sc in scans}) + 2 * len(scans)),
        "clocks": clocks,
    }
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the tensor-core precision modes (128^2 frames)")
    ap.add_argument("--copy-streams", type=int, default=1,
                    help="copy streams sharing each step's host-to-device upload in the e2e measurement")
    ap.add_argument("--workload", default="fermat", choices=["fermat", "raster256", "batch", "batch-small"])
    ap.add_argument("--frames", type=int, default=None,
                    help="frames of the scan (default: the workload's; fewer for small ncu captures; "
                         "raster256 rounds to a square raster)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        torch.distributed.init_process_group("nccl")
    if args.workload in ("batch", "batch-small"):
        run_batch(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
