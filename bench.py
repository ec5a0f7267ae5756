"""Benchmark: RAAR frame-iterations/s on one GB300 for the 10^4-frame raster
of 256^2 frames over a 3072^2 object (step 24 +-1 px, Poisson 10^8 photons
per frame, fixed probe, eps_a every step, eps_Q and eps_Delta every 10th),
with the fused frame kernel's HBM roofline fraction, an end-to-end figure
through the C ABI with host buffers, and the FP64 oracle timed on the host
cores as a reported CPU baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload raster256|fermat|batch|batch-small] [--no-mixed]
                  [--no-extra] [--copy-streams S]

The timed region runs the K steps with no timing hooks; a second pass of the
same steps with the library's per-launch CUDA events gives the per-kernel
breakdown and the frame kernel's average duration for the roofline.

Unless --no-extra is given, the line also carries "fermat": the 2500-frame
128^2 Fermat-spiral scan over a 1024^2 object (probe refinement every 2nd
step) measured the same way, with "mixed": its steps with the frame DFTs as
FP16 (per-frame scaled) and BF16x3 tensor-core contractions (128^2 frames).
--workload fermat makes that scan the headline instead.

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
RESIDUAL_EVERY = 10   # eps_Q and eps_Delta every 10th step; eps_a every step
FRAME_KERNEL = {"fermat": "raar_kernel<128>",
                "raster256": "raar_split256_kernel (256^2 frames as four 128^2 register transforms)"}
PROFILES = {"fermat": os.path.join(ROOT, "profiles", "raar_kernel_fermat128.txt"),
            "raster256": os.path.join(ROOT, "profiles", "raar_split256_raster256.txt")}
CSRC = os.path.join(ROOT, "paper_1602_01448_gb300", "csrc")


# Sources that make up each workload's frame-pass kernel: a committed ncu
# summary stays valid while these hash to the profiled version.
KERNEL_SOURCES = {
    "fermat": ["raar_kernel.cuh", "fft_frame.cuh", "tma.cuh", "sharp_common.cuh", "gen_twiddles.py",
               "raar_128_w0.cu"],
    "raster256": ["raar_split256.cuh", "raar_split256.cu", "fft_frame.cuh", "tma.cuh", "sharp_common.cuh",
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


def oracle_cores() -> int:
    """Host threads the oracle's transforms use (scipy.fft workers)."""
    import oracle as O
    return O.fft_workers()


def oracle_step_rate(scan, amps, n_frames: int, n_steps: int = 1):
    """FP64 oracle RAAR steps over the first n_frames frames of the scan (full
    object), with the probe update on the scan's cadence, as the GPU steps
    run them (Sec. 2.2 sequence): frame-iterations per second of host time."""
    import oracle as O
    pos = scan.pos[:n_frames]
    a = amps[:n_frames]
    t0 = time.perf_counter()
    O.raar_reconstruct(a, pos, scan.shape, scan.probe_init, scan.psi_init, n_steps, beta=0.75,
                       probe_every=scan.probe_every, record_metrics=False)
    dt = time.perf_counter() - t0
    return n_frames * n_steps / dt, dt


def oracle_amplitudes(scan, n_frames: int, seed: int = 5):
    """Noisy amplitudes of the first n_frames frames for the oracle arms,
    computed with the oracle's own forward model (the GPU arm computes its own
    with the library)."""
    import oracle as O
    import synth
    inten = O.forward_amplitudes(scan.obj, scan.probe, scan.pos[:n_frames]) ** 2
    return np.sqrt(synth.poisson_intensities(inten, scan.photons, seed))


def run_reference(args, rank):
    """The oracle as the reference arm: every step is one FP64 RAAR step (with
    the probe update on the scan's cadence) over a sample of the workload's
    frames, sized so that the K + W steps take about two minutes."""
    if rank != 0:
        return
    scan = make_scan(None, args.workload)
    per_frame_s = {64: 0.004, 128: 0.015, 256: 0.06}[scan.m]    # rough single-step cost per frame
    n = int(max(16, min(500, 120.0 / (per_frame_s * max(1, args.steps + args.warmup)))))
    n = min(n, scan.K)
    a = oracle_amplitudes(scan, n)
    steps_each = 2 if scan.probe_every else 1                    # one step with a probe update
    for _ in range(args.warmup):
        oracle_step_rate(scan, a, n, steps_each)
    times = []
    for _ in range(args.steps):
        _, dt = oracle_step_rate(scan, a, n, steps_each)
        times.append(dt / steps_each)
    ms = 1000.0 * float(np.mean(times))
    val = n / (ms / 1000.0)
    cores = oracle_cores()
    sample = (f"first {n} of {scan.K} frames of {scan.m}^2 per step, full {scan.shape[0]}^2 object, FP64 "
              f"NumPy/SciPy, transforms on {cores} threads"
              + (", probe update every 2nd step" if scan.probe_every else ""))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": scan.name, "sample": sample},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def timed_steps(plan, amp, steps, world, dev):
    """K RAAR steps between CUDA events on the launching stream, no timing
    hooks: the max over ranks of the elapsed milliseconds."""
    import torch
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        plan.raar_step(amp)
    e1.record(stream)
    torch.cuda.synchronize()
    return slowest_rank_ms(e0.elapsed_time(e1), world, dev)


def kernel_breakdown(S, plan, amp, steps):
    """The same steps again with the library's per-launch CUDA events on the
    launching stream: per kernel class (total ms over the steps, launches),
    and the whole pass's milliseconds with the hooks on."""
    import torch
    S.sharp_plan_set_profiling(plan.handle, True)
    S.sharp_plan_kernel_times(plan.handle)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        plan.raar_step(amp)
    torch.cuda.synchronize()
    wall = 1000.0 * (time.perf_counter() - t0)
    kt = S.sharp_plan_kernel_times(plan.handle)
    S.sharp_plan_set_profiling(plan.handle, False)
    return kt, wall


def frame_roofline(kt, m, K, peak):
    """HBM roofline of the fused frame kernel: 20 m^2 B per frame-iteration
    (state read 8, amplitudes read 4, state write 8) over its average launch
    duration."""
    frame_ms, frame_n = kt["frame"]
    t_frame = frame_ms / max(frame_n, 1) / 1000.0
    alg = 20.0 * m * m * K
    return alg, t_frame, alg / t_frame / 1e9


def time_mixed(S, scan, amp, psi0, w0, prec, steps, warmup, world, dev):
    """The same RAAR steps with the frame DFTs as tensor-core contractions
    (precision `prec`): throughput (hook-free timed steps), frame-kernel time
    (a second, profiled pass), its HBM fraction (20 m^2 B per frame) and its
    tensor-pipe rate.  The rate counts the dense-equivalent products issued:
    4 complex 128 x 128 x 128 products per 128^2 transform pair = 16 real
    ones, 2 * 128^3 flops each, four such pairs per 256^2 frame (its radix-2
    split into 128^2 sub-problems), three times for the BF16 three-term split;
    an FFT does ~2.3 MFLOP (128^2) of useful work per frame against these
    67 MFLOP, so the HBM fraction, not the tensor rate, is the figure of
    merit."""
    K, m = scan.K, scan.m
    plan = S.Plan(scan.pos, m, scan.shape, beta=0.75, probe_every=scan.probe_every,
                  residual_every=RESIDUAL_EVERY, device=dev, precision=prec)
    plan.raar_init(psi0, w0)
    for _ in range(warmup):
        plan.raar_step(amp)
    ms_total = timed_steps(plan, amp, steps, world, dev)
    kt, _ = kernel_breakdown(S, plan, amp, steps)
    plan.status()
    peak_hbm, _ = measured_peak_hbm()
    alg, t_frame, achieved = frame_roofline(kt, m, K, peak_hbm)
    terms = 3 if prec == "bf16x3" else 1
    flops = 16 * 2.0 * 128 ** 3 * (m // 128) ** 2 * terms * K
    peak_tc = measured_peak_tensor()
    met = plan.metrics.cpu().numpy().tolist()
    launches = sum(n for _, n in kt.values())
    out = {"precision": prec, "value": job_throughput(K, steps, world, ms_total), "unit": UNIT,
           "ms_per_step": ms_total / steps, "frame_kernel_ms": t_frame * 1000.0,
           "hbm": {"achieved": achieved, "peak": peak_hbm, "unit": "GB/s", "frac": achieved / peak_hbm},
           "tensor": {"achieved": flops / t_frame / 1e12, "peak": peak_tc, "unit": "TFLOP/s",
                      "frac": flops / t_frame / 1e12 / peak_tc if peak_tc else None,
                      "flops_per_launch": flops, "terms": terms,
                      "counts": "dense-equivalent products issued, not useful FFT work"},
           "gpu_launches": launches, "last_metrics": {"eps_a": met[0], "eps_q": met[1]}}
    plan.close()
    return out


def measure_scan(S, args, workload, frames, world, dev, local, rank, with_e2e=True, with_mixed=True,
                 with_cpu=True, steps=None):
    """One workload: hook-free timed steps (value), the per-kernel breakdown
    and roofline from a profiled pass, e2e with host buffers, the tensor-core
    modes (128^2) and the oracle on the host cores."""
    import torch
    import synth
    steps = args.steps if steps is None else steps
    scan = make_scan(frames, workload)
    K, m = scan.K, scan.m
    plan = S.Plan(scan.pos, m, scan.shape, beta=0.75, probe_every=scan.probe_every, residual_every=RESIDUAL_EVERY,
                  device=dev)
    obj = torch.as_tensor(scan.obj).to(torch.complex64).to(dev)
    probe_true = torch.as_tensor(scan.probe).to(torch.complex64).to(dev)
    amp = plan.forward_amplitudes(obj, probe_true)
    if workload == "fermat":
        inten = (amp.double() ** 2).cpu().numpy()
        amp_h = np.sqrt(synth.poisson_intensities(inten, scan.photons, 5)).astype(np.float32)
        amp = torch.as_tensor(amp_h).to(dev)
    else:
        amp = device_poisson(amp, scan.photons, 5)
    del obj, probe_true
    psi0 = torch.as_tensor(scan.psi_init).to(torch.complex64).to(dev)
    w0 = torch.as_tensor(scan.probe_init).to(torch.complex64).to(dev)
    plan.raar_init(psi0, w0)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        plan.raar_step(amp)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    ms_total = timed_steps(plan, amp, steps, world, dev)
    barrier()
    clocks = sampler.stop()
    metrics = plan.metrics.cpu().numpy().tolist()
    ms_step = ms_total / steps
    value = job_throughput(K, steps, world, ms_total)
    plan.status()

    # per-kernel breakdown and the frame kernel's launch duration (profiled pass)
    kt, prof_ms = kernel_breakdown(S, plan, amp, steps)
    peak, peak_kind = measured_peak_hbm()
    alg_bytes, t_frame, achieved = frame_roofline(kt, m, K, peak)
    launches_per_step = sum(n for _, n in kt.values()) / steps

    e2e = None
    if with_e2e:
        e2e = measure_e2e(plan, amp, args, world, dev, K)

    mixed = []
    if m in (128, 256) and with_mixed and not args.no_mixed:
        for prec in ("fp16s", "bf16x3"):
            mixed.append(time_mixed(S, scan, amp, psi0, w0, prec, steps, args.warmup, world, dev))
    plan.close()
    del amp
    torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and with_cpu and not args.no_cpu_baseline:
        # a bounded sample of the same steps: 500 frames of 256^2 (the
        # precision-study subset), all frames of smaller scans; two steps
        # (one with a probe update) when the scan refines its probe
        n = 500 if m == 256 else K
        n_steps = 2 if scan.probe_every else 1
        a_o = oracle_amplitudes(scan, n)
        rate, dt = oracle_step_rate(scan, a_o, n, n_steps)
        cores = oracle_cores()
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n_steps} FP64 RAAR step(s) (object update"
                         + (", probe update on the 2nd" if scan.probe_every else "")
                         + f") over {n} of {K} frames (full {scan.shape[0]}^2 object), {dt:.1f} s; "
                         f"transforms on {cores} threads (scipy.fft), the rest of the oracle single-threaded"}
    return {
        "scan": scan, "value": value, "ms_per_step": ms_step, "steps": steps, "clocks": clocks,
        "config": {"workload": scan.name, "frames": K, "frame": m, "object": list(scan.shape),
                   "beta": 0.75, "probe_every": scan.probe_every, "residual_every": RESIDUAL_EVERY,
                   "photons_per_frame": scan.photons, "parallelism": f"replicas{world}",
                   "l2": f"inputs larger than L2 (c {8 * K * m * m / 1e6:.0f} MB + a {4 * K * m * m / 1e6:.0f} MB per step)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": profiled_traffic(workload) if frames is None else None,
                     "kernel": FRAME_KERNEL[workload], "peak_kind": peak_kind,
                     "alg_bytes_per_launch": alg_bytes, "kernel_ms": t_frame * 1000.0,
                     "timing": "frame-kernel launches bracketed by CUDA events on the launching stream "
                               "(profiled pass of the same steps)"},
        "kernel_ms_per_step": {k: v[0] / steps for k, v in kt.items()},
        "profiled_pass_ms_per_step": prof_ms / steps,
        "gpu_launches": int(round(launches_per_step * steps)),
        "e2e": e2e, "mixed": mixed, "cpu_baseline": cpu,
        "last_metrics": {"eps_a": metrics[0], "eps_q": metrics[1]},
    }


def measure_e2e(plan, amp, args, world, dev, K):
    """End to end through the C ABI with host buffers: every step uploads its
    measured amplitudes from pinned host memory and reads the object back.
    The upload for step k+1 runs on its own stream while step k computes (two
    device buffers), and the object of step k is read back on a third stream
    from a device snapshot; every copy of the timed steps lies inside the
    timed region (the first upload starts after the start event, the end
    event waits for the last read-back)."""
    import torch
    stream = torch.cuda.current_stream()
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
    e2e_ms = slowest_rank_ms(f0.elapsed_time(f1) / e2e_steps, world, dev)
    out = {"value": world * K / (e2e_ms / 1000.0), "unit": UNIT,
           "h2d_bytes_per_step": int(amp.numel() * 4), "d2h_bytes_per_step": int(plan.psi.numel() * 8),
           "ms_per_step": e2e_ms, "copy_streams": n_up, "steps": e2e_steps}
    del amp_pin, amp_dev, psi_snap, psi_pin
    return out


def run_ours(args, rank, world):
    import torch
    import paper_1602_01448_gb300 as S

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    head = measure_scan(S, args, args.workload, args.frames, world, dev, local, rank)
    extra = None
    if args.workload == "raster256" and not args.no_extra and args.frames is None:
        # the 128^2 Fermat scan (probe refinement) and its tensor-core modes
        extra = measure_scan(S, args, "fermat", None, world, dev, local, rank, with_e2e=False, with_cpu=False,
                             steps=max(args.steps, 50))
    if rank != 0:
        return
    out = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": head["config"], "roofline": head["roofline"],
        "kernel_ms_per_step": head["kernel_ms_per_step"],
        "profiled_pass_ms_per_step": head["profiled_pass_ms_per_step"],
        "cpu_baseline": head["cpu_baseline"], "e2e": head["e2e"],
        "gpu_launches": head["gpu_launches"], "clocks": head["clocks"],
        "last_metrics": head["last_metrics"],
        # the same workload with the frame DFTs as tensor-core contractions
        # (FP16 per-frame scaled; BF16 three-term)
        "mixed": head["mixed"],
    }
    if extra is not None:
        out["fermat"] = {k: extra[k] for k in ("value", "ms_per_step", "steps", "config", "roofline",
                                               "kernel_ms_per_step", "gpu_launches", "clocks", "mixed",
                                               "last_metrics")}
        out["fermat"]["unit"] = UNIT
    print(json.dumps(out), flush=True)


def run_precision_study(args, rank, world):
    """Errors of the tensor-core precision modes on the 10^4-frame 256^2
    raster, against the FP64 oracle on a 500-frame subset (the first 5 rows of
    the raster, full 3072^2 object, Poisson 10^8 photons): the data projection
    P_a of one set of frames (per operator), and after `steps` RAAR steps from
    the scan's start the object against the oracle's object and eps_0 (Eq. 14)
    against the ground truth (final NRMSE).  FP32, BF16x3 and FP16S."""
    import torch
    import oracle as O
    import paper_1602_01448_gb300 as S
    import synth

    if rank != 0:
        return
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    full = synth.scan_large_raster()
    n = 500
    pos = full.pos[:n]
    shape, m = full.shape, full.m
    a = oracle_amplitudes(full, n, seed=9)
    steps = args.steps
    t0 = time.perf_counter()
    ref = O.raar_reconstruct(a, pos, shape, full.probe_init, full.psi_init, steps, beta=0.75,
                             psi_true=full.obj, record_metrics=False)
    t_oracle = time.perf_counter() - t0
    rng = np.random.default_rng(11)
    z = O.split(full.obj * np.exp(0.3j * rng.standard_normal(shape)), full.probe, pos[:50])
    pa_ref = O.data_project(z, a[:50])
    D = O.illumination(full.probe, pos, shape)
    vis = D > 1e-3 * D.max()
    out = {}
    for prec in ("fp32", "bf16x3", "fp16s"):
        plan = S.Plan(pos, m, shape, beta=0.75, residual_every=0, device=dev, precision=prec)
        zt = torch.as_tensor(z).to(torch.complex64).to(dev)
        at = torch.as_tensor(a).to(torch.float32).to(dev)
        p50 = S.Plan(pos[:50], m, shape, precision=prec, device=dev)
        got, _ = p50.fourier_project(zt, at[:50].contiguous())
        pa_err = float(np.linalg.norm(got.cpu().numpy() - pa_ref) / np.linalg.norm(pa_ref))
        p50.close()
        plan.raar_init(torch.as_tensor(full.psi_init).to(torch.complex64).to(dev),
                       torch.as_tensor(full.probe_init).to(torch.complex64).to(dev))
        for _ in range(steps):
            plan.raar_step(at, metrics=False)
        plan.status()
        e0 = plan.solution_error(plan.psi, torch.as_tensor(full.obj).to(torch.complex64).to(dev),
                                 torch.as_tensor(full.probe).to(torch.complex64).to(dev))[0].item()
        psi = plan.psi.cpu().numpy().astype(np.complex128)
        obj_err = float(np.linalg.norm((psi - ref["psi"])[vis]) / np.linalg.norm(ref["psi"][vis]))
        out[prec] = {"p_a_rel_l2": pa_err, "object_rel_l2_vs_oracle": obj_err, "eps_0": e0}
        plan.close()
    print(json.dumps({"study": "precision", "workload": f"{full.name} subset: first {n} frames",
                      "steps": steps, "oracle_eps_0": ref["history"][-1]["eps_0"], "oracle_s": t_oracle,
                      "p_a_frames": 50, "modes": out}), flush=True)


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

    for _ in range(max(args.warmup, 8)):        # covers the autotuner's candidate steps (at most 6)
        batch.step()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ms_total = timed(batch.step, args.steps)
    clocks = sampler.stop()
    batch.status()
    ms_total = slowest_rank_ms(ms_total, world, dev)
    ms_step = ms_total / args.steps

    # the tuned launch shapes against the library's defaults (one block per
    # SM, 8 rows per round trip, 4 for 256^2, 2 us stagger): same steps again
    sizes = sorted({sc.m for sc in scans})
    shapes = {str(m): list(batch.tuned_shape(m)) for m in sizes}
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    for m in sizes:
        batch.set_shape(m, sms, 4 if m == 256 else 8, 2000)
    for _ in range(3):
        batch.step()
    ms_default = slowest_rank_ms(timed(batch.step, args.steps), world, dev) / args.steps
    batch.status()

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
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        sc = scans[0]
        n = min(sc.K, 300)
        a_o = oracle_amplitudes(sc, n)
        rate, dt = oracle_step_rate(sc, a_o, n, 1)
        cores = oracle_cores()
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"one FP64 RAAR step + object update over {n} frames of {sc.m}^2 "
                         f"(first scan of the batch), {dt:.1f} s; transforms on {cores} threads (scipy.fft)"}
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
                   "parallelism": f"replicas{world}", "tuned_shape": shapes,
                   "l2": f"inputs larger than L2 ({alg_bytes * 0.6 / 1e9:.1f} GB of state + amplitudes read per step)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "whole step (all launches of sharp_batch_step)",
                     "peak_kind": peak_kind, "alg_bytes_per_launch": alg_bytes, "kernel_ms": ms_step},
        "one_by_one": {"ms_per_step": ms_single, "value": total / (ms_single / 1000.0),
                       "speedup_of_batch": ms_single / ms_step},
        "autotuner": {"shape": "[grid, rows per round trip, stagger ns] per frame size",
                      "default_ms_per_step": ms_default, "tuned_ms_per_step": ms_step,
                      "gain": ms_default / ms_step},
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
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the tensor-core precision modes")
    ap.add_argument("--copy-streams", type=int, default=1,
                    help="copy streams sharing each step's host-to-device upload in the e2e measurement")
    ap.add_argument("--workload", default="raster256",
                    choices=["raster256", "fermat", "batch", "batch-small", "precision256"])
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the 128^2 Fermat scan (and its tensor-core modes) after the headline workload")
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
    elif args.workload == "precision256":
        run_precision_study(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
