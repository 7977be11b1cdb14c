#!/usr/bin/env python3
"""Throughput of the TRDMD forward cascade on GB300.

Workload (per GPU): one 512x512 speckled image (L = 1), T = 5 stages of 48
zero-mean 7x7 filters with 63-RBF influence functions, plain FP32, fused stage
kernel -- one "step" is the whole T-stage forward of that image.  With N GPUs
(torchrun), every rank runs its own image (independent problems, no
collective on the data path): weak scaling.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line (rank 0).  `value` is Mpixel/s over all ranks with the
inputs resident in HBM (L2 flushed between steps by a 256 MiB write, outside
the step's events); `e2e` is the same metric through the C ABI with the input
copied from pinned host memory and u_T copied back inside the timed region.
`--impl reference` times the FP64 CPU oracle on the host cores instead (a
bounded row band of the same image per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpixel/s fwd & fwd+bwd (7x7x48, T=5), plain FP32 vs batched/mixed precision"
H = W = 512
KS, NK, T, L = 7, 48, 5, 1
CFG_ID = 2
# Algorithmic work of one stage per pixel: filter bank 2*N_k*k^2, adjoint
# 2*N_k*k^2, phi as the method's full sum 2*N_k*N_rbf (one FMA per RBF term;
# the exps are on top), prox ~12 flops.
FLOPS_PER_PX_STAGE = 2 * NK * KS * KS * 2 + 2 * NK * 63 + 12
CONFIG = {"workload": "TRDMD forward, 1 x 512x512 per GPU, 7x7x48, 63 RBF, T=5, L=1, "
                      "fused FP32 stage kernel",
          "H": H, "W": W, "images_per_gpu": 1, "ksize": KS, "nfilt": NK, "nrbf": 63, "T": T,
          "looks": L, "l2": "flushed between steps (256 MiB write outside the events)"}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# DRAM bytes (read + write) per launch of the stage kernel at this workload,
# from one ncu capture (profiles/fused_stage_fwd_7x7x48_512x512.md), valid only
# for the kernel sources it was taken on (their hash is checked at run time).
_TRAFFIC = {"sources_sha256_16": "20c231ed885ecf70", "bytes_per_launch": 2205440}


def _kernel_sources_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("fused_fwd.cuh", "common.cuh", "args.cuh"):
        with open(os.path.join(ROOT, "paper_1702_07482_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _measured_traffic():
    try:
        if _kernel_sources_hash() == _TRAFFIC["sources_sha256_16"]:
            return _TRAFFIC["bytes_per_launch"]
    except OSError:
        pass
    return None


def _fp32_peak_tflops(sm_mhz: float, n_sm: int) -> float:
    # 128 FP32 lanes per SM, one FMA (2 flops) per lane per clock
    return n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """Samples nvidia-smi during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _inputs():
    import numpy as np
    import synth
    p = synth.params(T, KS, NK, seed=synth.seed_for(CFG_ID, 0, "params"))
    p = p.astype(np.float32).astype(np.float64)
    _, f = synth.single_image(H, W, L, CFG_ID, index=0)
    return p, f.astype(np.float32).astype(np.float64)


def _cpu_oracle_rate(p, f, rows: int):
    """Mpixel/s of the FP64 oracle on a band of `rows` image rows (T stages)."""
    import oracle
    band = f[:rows].copy()
    t0 = time.perf_counter()
    oracle.forward(band, p)
    dt = time.perf_counter() - t0
    return rows * W / dt / 1e6, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    p, f = _inputs()
    # size the row band so that one step takes about 1-4 s
    rows = 8
    _, dt = _cpu_oracle_rate(p, f, rows)
    rows = int(max(4, min(H, rows * 2.0 / max(dt, 1e-3))))
    for _ in range(args.warmup):
        _cpu_oracle_rate(p, f, rows)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.forward(f[:rows].copy(), p)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    value = rows * W / (ms / 1e3) / 1e6
    cores = oracle.get_threads()
    sample = f"rows 0..{rows - 1} of the 512x512 image (all T={T} stages, 7x7x48) per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mpixel/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": CONFIG,
        "cpu_baseline": {"value": value, "unit": "Mpixel/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "Mpixel/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1702_07482_gb300 import binding, build, ops
    build.build()
    binding.load()

    p, f = _inputs()
    m = ops.Model.create(p.filters, p.rbf_w, p.lam, p.mu0, p.delta, p.gamma, device=dev)
    f_dev = torch.tensor(f, dtype=torch.float32, device=dev).unsqueeze(0).contiguous()
    u_dev = torch.empty_like(f_dev)
    prm = m.params()
    ws_bytes = binding.tnrd_workspace_size(binding.OP_FORWARD, prm, 1, H, W, W, 0, 0)
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        binding.tnrd_forward(prm, 1, H, W, W, f_dev, u_dev, 0, 0, ws, ws_bytes, sp)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(max(args.warmup, 3)):
        step()
    barrier()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    barrier()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)          # evict the image from L2 between steps
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in evs]

    # end to end through the C ABI: pinned host input -> device -> stage
    # cascade -> pinned host output, all inside the events
    f_host = torch.tensor(f, dtype=torch.float32).unsqueeze(0).contiguous().pin_memory()
    u_host = torch.empty_like(f_host).pin_memory()
    e2e_evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    for _ in range(3):
        f_dev.copy_(f_host, non_blocking=True)
        step()
        u_host.copy_(u_dev, non_blocking=True)
    barrier()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        e2e_evs[i][0].record(stream)
        f_dev.copy_(f_host, non_blocking=True)
        step()
        u_host.copy_(u_dev, non_blocking=True)
        e2e_evs[i][1].record(stream)
    barrier()
    clocks = sampler.stop()
    e2e_ms = [a.elapsed_time(b) for a, b in e2e_evs]

    ms = statistics.mean(step_ms)
    ms_e2e = statistics.mean(e2e_ms)
    # every rank ran its own image: all ranks' pixels over the slowest rank's time
    from paper_1702_07482_gb300.shard import global_rate
    value, ms = global_rate(H * W, ms)
    e2e_value, ms_e2e = global_rate(H * W, ms_e2e)
    out = None
    if rank == 0:
        peaks, src = _peaks()
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        sm_max = float(peaks.get("sm_max_mhz", 2070.0))
        peak_tf = _fp32_peak_tflops(sm_max, n_sm)
        launch_ms = ms / T   # T launches of the stage kernel per step, back to back
        achieved_tf = H * W * FLOPS_PER_PX_STAGE / (launch_ms / 1e3) / 1e12
        traffic = _measured_traffic()
        cpu = None
        if not args.no_cpu_baseline:
            import oracle
            oracle.build()
            rows = 16
            rate, dt = _cpu_oracle_rate(p, f, rows)
            rows = int(max(8, min(H, rows * 12.0 / max(dt, 1e-3))))
            rate, dt = _cpu_oracle_rate(p, f, rows)
            cpu = {"value": rate, "unit": "Mpixel/s", "cores": oracle.get_threads(),
                   "kind": "oracle",
                   "sample": f"rows 0..{rows - 1} of the 512x512 image, all T={T} stages "
                             f"({dt:.1f} s)"}
        out = {
            "metric": METRIC, "value": value, "unit": "Mpixel/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": CONFIG,
            "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": peak_tf,
                         "unit": "TFLOP/s", "frac": achieved_tf / peak_tf,
                         "traffic": traffic,
                         "kernel": "fused_stage_fwd<7,48,TH>",
                         "peak_source": f"derived: {n_sm} SMs x 128 FP32 lanes x 2 x "
                                        f"{sm_max:.0f} MHz ({src} sm_max_mhz)",
                         "flops_per_px_stage": FLOPS_PER_PX_STAGE},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "Mpixel/s",
                    "h2d_bytes_per_step": int(f_host.numel() * 4),
                    "d2h_bytes_per_step": int(u_host.numel() * 4)},
            "gpu_launches": args.steps * T,
            "clocks": clocks,
        }
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if out is not None:
        print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
