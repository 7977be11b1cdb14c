#!/usr/bin/env python3
"""Throughput of the TRDMD despeckling cascade on GB300.

Default workload (per GPU): one 512x512 speckled image (L = 1), T = 5 stages of
48 zero-mean 7x7 filters with 63-RBF influence functions, plain FP32, fused
stage kernel -- one "step" is the whole T-stage forward of that image.  With N
GPUs (torchrun), every rank runs its own image (independent problems, no
collective on the data path): weak scaling.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload fwd512|fwd512_unfused|fwd512_tf32x3|small128|batched|
                              batched_tf32|batched_bf16|batched_tf32x3|train|train_tf32|
                              train_bf16|train_tf32x3|train_tc|fit|fit_tf32|fwd512_gauss|
                              fwd512_proj|
                              quality|mixed_tf32|mixed_bf16|mixed_fp32|mixed_tf32x3]
                  [--no-cpu-baseline] [--no-accuracy] [--no-alt]

The other workloads (one GPU) measure the rest of the table with the same
contract: fwd512_unfused (three kernels per stage), small128 (1 x 128^2,
5x5x24), batched (64 images of 256-1024 px per side, four parameter sets, one
persistent launch per step; batched_tf32 / batched_bf16 the same batch with the
tensor-core stage, one launch per stage), train (32 x 180^2 crops, forward +
backward),
fit (one Adam iteration of joint training on the same crops), fwd512_gauss /
fwd512_proj (the 512^2 forward with TNRD's Gaussian-denoising reaction term on
sigma = 25 noise, and with the explicit step plus projection), quality (the
Sec. 4 quality indexes of 16 x 2048^2 image triplets; ALU roofline),
mixed_tf32 / mixed_bf16 / mixed_fp32 (16 x 2048^2, L = 2, T = 8, tensor-core
TF32 and BF16 vs plain FP32; the line adds the path's error against the FP64
oracle); the *_tf32x3 workloads run the split-TF32 tensor-core stage (FP32
accuracy), train_tf32 / train_bf16 / fit_tf32 the training step with a
tensor-core forward (the backward FP32).  On one GPU the default line also
carries `fp32_accurate_tensor_core`: the same image through the split-TF32
stage, timed the same way, with its error against the same oracle run
(`--no-alt` leaves it out); the headline `value` stays the CUDA-core FP32 stage.

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
# Quality indexes per pixel, by their definitions: SSIM window means of x and y
# (2 x 121 FMA = 484 flops) and second moments E[x^2], E[y^2], E[xy] (3 x 121 x
# (mul + FMA) = 1089), SSIM from the five statistics (21), squared error (3), two
# 5-tap Laplacians and the five edge-correlation sums (18), ratio image with its two
# sums (4), coefficient-of-variation sums (3).
QUALITY_FLOPS_PER_PX = 484 + 1089 + 21 + 3 + 18 + 4 + 3
CONFIG = {"workload": "TRDMD forward, 1 x 512x512 per GPU, 7x7x48, 63 RBF, T=5, L=1, "
                      "fused FP32 stage kernel",
          "H": H, "W": W, "images_per_gpu": 1, "ksize": KS, "nfilt": NK, "nrbf": 63, "T": T,
          "looks": L, "data_term": "idiv",
          "l2": "flushed between steps (256 MiB write outside the events)"}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# DRAM bytes (read + write) per launch of the fused stage kernel at the 512 x 512
# workload, from one ncu capture of that kernel (dram__bytes_read.sum +
# dram__bytes_write.sum of a steady-state launch), valid only for the kernel that capture measured and the sources it was taken
# on (the kernel name and the sources' hash are checked at run time).
_TRAFFIC = {"kernel": "fused_pair2_fwd<7,48,37> tiles 33x58 (border rows 27), tma staging",
            "sources_sha256_16": "088e8ec313740543", "bytes_per_launch": 2276096}


def _kernel_sources_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("fused_fwd.cuh", "fused_pair.cuh", "tile_stage.cuh", "common.cuh", "args.cuh"):
        with open(os.path.join(ROOT, "paper_1702_07482_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _measured_traffic(kernel: str):
    try:
        if (kernel == _TRAFFIC["kernel"] and
                _kernel_sources_hash() == _TRAFFIC["sources_sha256_16"]):
            return _TRAFFIC["bytes_per_launch"]
    except OSError:
        pass
    return None


def _fp32_peak_tflops(sm_mhz: float, n_sm: int) -> float:
    # 128 FP32 lanes per SM, one FMA (2 flops) per lane per clock
    return n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12


class NvmlClocks:
    """Read-only SM clock and clock-event-reason samples through NVML (the
    driver's libnvidia-ml, via ctypes), taken every ~1 ms by a host thread;
    only the samples that fall inside the marked timed windows are kept."""

    SM = 1   # NVML_CLOCK_SM
    # clock event reason bits (nvmlClocksEventReason*)
    BITS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
            0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, dev):
        import ctypes
        self.ok = False
        self.samples = []
        self.windows = []
        self._stop = threading.Event()
        self._t = None
        try:
            L = ctypes.CDLL("libnvidia-ml.so.1")
            if L.nvmlInit_v2() != 0:
                return
            self.L = L
            h = ctypes.c_void_p()
            import torch
            pr = torch.cuda.get_device_properties(dev)
            bus = getattr(pr, "pci_bus_id", None)
            rc = 1
            if bus is not None:
                pci = f"{getattr(pr, 'pci_domain_id', 0):08x}:{bus:02x}:{pr.pci_device_id:02x}.0"
                rc = L.nvmlDeviceGetHandleByPciBusId_v2(pci.encode(), ctypes.byref(h))
            if rc != 0:
                rc = L.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(dev.index or 0), ctypes.byref(h))
            if rc != 0:
                return
            self.h = h
            self.reasons_fn = getattr(L, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                L.nvmlDeviceGetCurrentClocksThrottleReasons
            mx = ctypes.c_uint()
            self.sm_max = (float(mx.value) if L.nvmlDeviceGetMaxClockInfo(h, self.SM, ctypes.byref(mx))
                           == 0 else None)
            self.ok = True
        except (OSError, AttributeError):
            self.ok = False

    def _read(self):
        import ctypes
        c = ctypes.c_uint()
        r = ctypes.c_ulonglong()
        while not self._stop.is_set():
            t = time.perf_counter()
            if self.L.nvmlDeviceGetClockInfo(self.h, self.SM, ctypes.byref(c)) == 0:
                rr = r.value if self.reasons_fn(self.h, ctypes.byref(r)) == 0 else 0
                self.samples.append((t, float(c.value), rr))
            time.sleep(0.001)

    def start(self):
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def mark(self, t0, t1):
        self.windows.append((t0, t1))

    def stop(self):
        self._stop.set()
        if self._t:
            self._t.join(timeout=2)
        inside = [(c, r) for (t, c, r) in self.samples
                  if any(a <= t <= b for a, b in self.windows)]
        reasons = sorted({nm for _, r in inside for bit, nm in self.BITS.items() if r & bit})
        return {"sm_mhz": statistics.median(c for c, _ in inside) if inside else None,
                "sm_max_mhz": self.sm_max, "reasons": reasons, "samples": len(inside),
                "source": "NVML, read-only, ~1 ms period; only samples inside the timed "
                          "regions (device-timed steps and end-to-end steps)",
                "window_ms": round(1e3 * sum(b - a for a, b in self.windows), 3)}


class ClockSampler:
    """Samples nvidia-smi during the timed region (used when NVML cannot be read)."""

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


def _p32(p):
    import numpy as np
    return p.astype(np.float32).astype(np.float64)


# Algorithmic flops per pixel-stage of the backward at 7x7x48 (fwd: FLOPS_PER_PX_STAGE):
# convolutions z = K u, b = K d, the adjoint of c and the two filter-gradient
# correlations (5 x 2 N_k k^2), phi, phi' and the RBF-weight gradient
# (3 x 2 N_k N_rbf), ~20 for y, x and d.
BWD_FLOPS_PER_PX_STAGE = 5 * 2 * NK * KS * KS + 3 * 2 * NK * 63 + 20


class Workload:
    """One benchmark workload: device-resident step, end-to-end step, and the
    numbers the JSON line needs.  Subclasses set the attributes in setup()."""
    name = ""
    config = {}
    px = 0                 # pixels processed per step (per rank)
    launches = 0           # our kernel launches per step
    flops = 0.0            # algorithmic flops per step
    kernel = ""
    h2d = 0
    d2h = 0
    traffic = None

    def __init__(self, dev):
        self.dev = dev

    def step(self):
        raise NotImplementedError

    def e2e(self):
        raise NotImplementedError

    def cpu_baseline(self):
        return None


def _rows_rate(fn, rows0, target_s, max_rows):
    """Runs fn(rows) growing the row count until one call takes ~target_s."""
    rows = rows0
    dt = 0.0
    for _ in range(4):
        t0 = time.perf_counter()
        fn(rows)
        dt = time.perf_counter() - t0
        if dt >= 0.5 * target_s or rows >= max_rows:
            break
        rows = int(min(max_rows, max(rows + 1, rows * target_s / max(dt, 1e-3))))
    return rows, dt


def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() == "Model name":
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def _oracle_baseline(fn, rows0, max_rows, width, what, full=None):
    """The FP64 oracle's rate on the host cores, all cores and one thread.
    fn(rows) runs the oracle on the first `rows` rows of the workload's image;
    `full` = (pixels, seconds) of a timed all-core oracle run over a whole image
    (the accuracy check's), used as the all-core sample when given."""
    import oracle
    oracle.build()
    n = oracle.get_threads()
    if full is not None:
        px, dt = full
        v_all, s_all = px / dt / 1e6, f"the whole {what}, all stages ({dt:.1f} s)"
    else:
        rows, dt = _rows_rate(fn, rows0, 12.0, max_rows)
        v_all, s_all = rows * width / dt / 1e6, f"rows 0..{rows - 1} of {what}, all stages ({dt:.1f} s)"
    oracle.set_threads(1)
    try:
        rows1, dt1 = _rows_rate(fn, max(1, rows0 // 4), 8.0, max_rows)
    finally:
        oracle.set_threads(n)
    return {"value": v_all, "unit": "Mpixel/s", "cores": n, "kind": "oracle", "sample": s_all,
            "value_1thread": rows1 * width / dt1 / 1e6,
            "sample_1thread": f"rows 0..{rows1 - 1} of {what}, all stages, 1 thread ({dt1:.1f} s)",
            "cpu_model": _cpu_model(), "nproc": os.cpu_count()}


def _accuracy(got, ref, what):
    """max |du| and PSNR of a whole GPU result against the FP64 oracle's."""
    import numpy as np
    d = np.asarray(got, np.float64) - np.asarray(ref, np.float64)
    mse = float((d ** 2).mean())
    return {"vs": "FP64 oracle", "pixels": int(d.size), "image": what,
            "max_abs": float(np.abs(d).max()),
            "psnr_db": float(10 * np.log10(255.0 ** 2 / max(mse, 1e-30))),
            "scale": "[0, 255] intensities"}


def _timed_oracle_forward(f, p):
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    u = oracle.forward(f, p)
    return u, time.perf_counter() - t0


class Fwd(Workload):
    def __init__(self, dev, H=512, W=512, ks=KS, nk=NK, T_=T, algo="fused", cfg=CFG_ID,
                 data_term=0):
        super().__init__(dev)
        import numpy as np
        import torch
        import synth
        from paper_1702_07482_gb300 import binding, ops
        self.Hh, self.Ww, self.T = H, W, T_
        self.p = _p32(synth.params(T_, ks, nk, seed=synth.seed_for(cfg, 0, "params")))
        self.p.dterm = data_term
        if data_term == 1:
            # TNRD Gaussian denoising: additive N(0, 25^2) noise, small reaction weights
            self.p.lam = 0.1 * np.arange(1, T_ + 1, dtype=np.float64)
            clean = synth.clean_image(H, W, synth.seed_for(cfg, 0, "image"))
            f = synth.gaussian_noise(clean, 25.0, synth.seed_for(cfg, 0, "noise"))
        else:
            _, f = synth.single_image(H, W, L, cfg, index=0)
        self.f = f.astype(np.float32).astype(np.float64)
        m = ops.Model.create(self.p.filters, self.p.rbf_w, self.p.lam, device=dev,
                             data_term=data_term, proj_c=1.0)
        self.prm = m.params()
        self.model = m
        self.P = ops.pitch_for(W)
        self.f_dev = ops.to_pitched(torch.tensor(self.f, dtype=torch.float32, device=dev))
        self.u_dev = torch.empty_like(self.f_dev)
        self.algo = binding.ALGO[algo]
        self.ws_bytes = binding.tnrd_workspace_size(binding.OP_FORWARD, self.prm, 1, H, W, self.P,
                                                    0, self.algo)
        self.ws = torch.empty(max(self.ws_bytes, 1), dtype=torch.uint8, device=dev)
        self.sp = torch.cuda.current_stream(dev).cuda_stream
        self.f_host = self.f_dev.cpu().pin_memory()
        self.u_host = torch.empty_like(self.f_host).pin_memory()
        self.px = H * W
        self.launches = T_ * (3 if algo == "unfused" else 1)
        if algo in TENSOR_RATIO:
            self.tensor_dtype = algo
            self.dtype = ("f32 (split TF32 tensor-core products)" if algo == "tf32x3"
                          else f"{algo} operands, f32 accumulate")
        fl = 2 * nk * ks * ks * 2 + 2 * nk * 63 + 12
        self.flops = float(H * W) * T_ * fl
        self.flops_per_px_stage = fl
        self.kernel = binding.tnrd_forward_kernel(self.prm, 1, H, W, self.algo)
        self.h2d = self.d2h = int(self.f_host.numel() * 4)
        self.traffic = (_measured_traffic(self.kernel)
                        if (algo == "fused" and H == 512 and data_term == 0) else None)
        noise = {0: f"L={L}", 1: "Gaussian sigma=25", 2: f"L={L}"}[data_term]
        dterm = {0: "", 1: ", TNRD Gaussian-denoising reaction (Sec. 2.2.1)",
                 2: ", explicit step with projection max(u, 1) (Eq. diffusion_backP)"}[data_term]
        kdesc = (f"{algo} FP32 stage kernel" + ("" if algo == "fused" else "s")
                 if algo in ("fused", "unfused") else
                 f"tensor-core stage ({PREC_TEXT[algo]}; phi and prox FP32)")
        self.config = {"workload": f"TRDMD forward, 1 x {H}x{W} per GPU, {ks}x{ks}x{nk}, 63 RBF, "
                                   f"T={T_}, {noise}, {kdesc}" + dterm,
                       "H": H, "W": W, "images_per_gpu": 1, "ksize": ks, "nfilt": nk,
                       "nrbf": 63, "T": T_, "looks": L if data_term != 1 else None,
                       "data_term": ["idiv", "gauss", "proj"][data_term],
                       "l2": "flushed between steps (256 MiB write outside the events)"}

    def step(self):
        from paper_1702_07482_gb300 import binding
        binding.tnrd_forward(self.prm, 1, self.Hh, self.Ww, self.P, self.f_dev, self.u_dev, 0,
                             self.algo, self.ws, self.ws_bytes, self.sp)

    def e2e(self):
        self.f_dev.copy_(self.f_host, non_blocking=True)
        self.step()
        self.u_host.copy_(self.u_dev, non_blocking=True)

    def accuracy(self):
        """u_T of the whole image against the FP64 oracle (whose run, timed on
        all host cores, is also the all-core CPU baseline sample)."""
        import torch
        self.step()
        torch.cuda.synchronize()
        got = self.u_dev[0, :, :self.Ww].double().cpu().numpy()
        u, dt = _timed_oracle_forward(self.f, self.p)
        self._full = (self.Hh * self.Ww, dt)
        self.ref_uT = u[-1]
        return _accuracy(got, u[-1], f"{self.Hh}x{self.Ww} image (u_T)")

    def cpu_baseline(self):
        import oracle
        band = lambda r: oracle.forward(self.f[:r].copy(), self.p)
        return _oracle_baseline(band, 8, self.Hh, self.Ww, f"the {self.Hh}x{self.Ww} image",
                                getattr(self, "_full", None))


class Batched(Workload):
    def __init__(self, dev, n=64, lo=256, hi=1024, T_=T, cfg=3, algo="fused"):
        super().__init__(dev)
        import numpy as np
        import torch
        import synth
        from paper_1702_07482_gb300 import binding as B
        from paper_1702_07482_gb300 import ops
        looks = (1, 2, 4, 8)
        self.T = T_
        self.sizes = synth.uneven_batch(n, lo, hi, cfg, looks)
        self.params = [_p32(synth.params(T_, KS, NK, seed=synth.seed_for(cfg, s, "params")))
                       for s in range(len(looks))]
        self.models = [ops.Model.create(p.filters, p.rbf_w, p.lam, device=dev) for p in self.params]
        offs, tot = [], 0
        for (Hh, Ww, Lk) in self.sizes:
            offs.append(tot)
            tot += Hh * ops.pitch_for(Ww)
        self.f_host = torch.zeros(tot, dtype=torch.float32).pin_memory()
        self.fs = []
        for i, (Hh, Ww, Lk) in enumerate(self.sizes):
            _, f = synth.single_image(Hh, Ww, Lk, cfg, index=i)
            f = f.astype(np.float32)
            P = ops.pitch_for(Ww)
            view = self.f_host[offs[i]:offs[i] + Hh * P].view(Hh, P)
            view[:, :Ww] = torch.from_numpy(f)
            if i == 0:
                self.fs.append(f.astype(np.float64))
        self.f_dev = self.f_host.to(dev)
        self.u_dev = torch.zeros_like(self.f_dev)
        self.u_host = torch.empty_like(self.f_host).pin_memory()
        imgs = []
        for i, (Hh, Ww, Lk) in enumerate(self.sizes):
            P = ops.pitch_for(Ww)
            imgs.append(B.tnrd_image(self.f_dev[offs[i]:].data_ptr(), self.u_dev[offs[i]:].data_ptr(),
                                     Hh, Ww, P, looks.index(Lk)))
        self.sp = torch.cuda.current_stream(dev).cuda_stream
        self.plan = B.Plan(imgs, [m.params() for m in self.models], algo=B.ALGO[algo],
                           autotune=True, stream=self.sp)
        self.px = sum(Hh * Ww for (Hh, Ww, _) in self.sizes)
        self.launches = self.plan.launches
        self.flops = float(self.px) * T_ * FLOPS_PER_PX_STAGE
        self.flops_per_px_stage = FLOPS_PER_PX_STAGE
        self.algo = algo
        if algo != "fused":
            self.dtype = ("f32 (split TF32 tensor-core products)" if algo == "tf32x3"
                          else f"{algo} operands, f32 accumulate")
            self.tensor_dtype = algo
        sched = ("batch_persistent_fwd" if self.launches == 1 else
                 "batch_pair2_fwd" if self.plan.tile_width == 64 - 2 * (KS // 2) else "batch_stage_fwd")
        self.kernel = (f"{sched}<7,48,{self.plan.tile_height}>" if algo == "fused" else
                       f"tc_batch_fwd<7,48,{(self.plan.tile_height + 2 * (KS // 2)) // 16},{algo}> "
                       f"(tcgen05 {algo.upper()} filter bank and "
                       f"adjoint, FP32 phi/prox; one launch per stage)")
        self.h2d = self.d2h = int(self.f_host.numel() * 4)
        self.config = {"workload": f"TRDMD batched forward, {n} images with sides U[{lo},{hi}] "
                                   f"({self.px / 1e6:.1f} Mpx), L in {{1,2,4,8}} with one "
                                   f"7x7x48 63-RBF parameter set each, T={T_}, " +
                                   (f"{'one persistent launch' if self.launches == 1 else 'one launch per stage'} "
                                    f"per step (CUDA graph), autotuned tile geometry and schedule "
                                    f"(tiles {self.plan.tile_height}x{self.plan.tile_width})" if algo == "fused" else
                                    f"{algo.upper()} tensor-core stage, one launch per stage over "
                                    f"all images' tiles (CUDA graph)"),
                       "images": n, "pixels": self.px, "ksize": KS, "nfilt": NK, "nrbf": 63,
                       "T": T_, "tile_height": self.plan.tile_height,
                       "l2": f"inputs ({self.h2d / 2 ** 20:.0f} MiB) larger than L2"}

    def step(self):
        self.plan.forward(self.sp)

    def accuracy(self):
        """u_T of the whole image 0 of the batch against the FP64 oracle."""
        import torch
        from paper_1702_07482_gb300 import ops
        self.step()
        torch.cuda.synchronize()
        Hh, Ww, Lk = self.sizes[0]
        P = ops.pitch_for(Ww)
        got = self.u_dev[:Hh * P].view(Hh, P)[:, :Ww].double().cpu().numpy()
        u, dt = _timed_oracle_forward(self.fs[0], self.params[0])
        self._full = (Hh * Ww, dt)
        return _accuracy(got, u[-1], f"image 0 of the batch, {Hh}x{Ww}, L={Lk} (u_T)")

    def e2e(self):
        self.f_dev.copy_(self.f_host, non_blocking=True)
        self.step()
        self.u_host.copy_(self.u_dev, non_blocking=True)

    def cpu_baseline(self):
        import oracle
        f0 = self.fs[0]
        p0 = self.params[0]
        band = lambda r: oracle.forward(f0[:r].copy(), p0)
        return _oracle_baseline(band, 8, f0.shape[0], f0.shape[1],
                                f"image 0 ({f0.shape[0]}x{f0.shape[1]})",
                                getattr(self, "_full", None))


class Train(Workload):
    """Training step: forward cascade with its checkpoints u_0..u_T (FP32 stage
    kernels, or the TF32 / BF16 tensor-core stage with algo), then the FP32
    backward of every stage."""

    def __init__(self, dev, n=32, S=180, T_=T, cfg=4, algo="fused", bwd_algo="fused"):
        super().__init__(dev)
        import numpy as np
        import torch
        import synth
        from paper_1702_07482_gb300 import binding as B
        from paper_1702_07482_gb300 import ops
        self.T, self.n, self.S, self.algo, self.bwd_algo = T_, n, S, algo, bwd_algo
        self.p = _p32(synth.params(T_, KS, NK, seed=synth.seed_for(cfg, 0, "params")))
        rank = int(os.environ.get("RANK", "0"))      # each rank its own crops (weak scaling)
        pairs = [synth.single_image(S, S, 1, cfg, index=rank * n + i) for i in range(n)]
        self.clean = np.stack([c for c, _ in pairs]).astype(np.float32)
        self.f = np.stack([f for _, f in pairs]).astype(np.float32)
        self.m = ops.Model.create(self.p.filters, self.p.rbf_w, self.p.lam, device=dev)
        self.P = ops.pitch_for(S)
        self.f_dev = ops.to_pitched(torch.tensor(self.f, device=dev))
        self.c_dev = ops.to_pitched(torch.tensor(self.clean, device=dev))
        self.f_host = self.f_dev.cpu().pin_memory()
        self.c_host = self.c_dev.cpu().pin_memory()
        self.u_all = torch.empty((T_ + 1,) + tuple(self.f_dev.shape), device=dev)
        self.ws_bytes = ops.workspace_size(self.m, n, S, S, self.P, 1, op=B.OP_BACKWARD,
                                           algo=bwd_algo)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        self.g_host = torch.empty(self.m.filters.numel() + self.m.rbf_w.numel() + T_,
                                  dtype=torch.float32).pin_memory()
        self.grads = None
        self.px = n * S * S
        self.launches = T_ + T_ * 5   # forward stages; prep, zb, adj, dk, reduce per stage
        self.flops = float(self.px) * T_ * (FLOPS_PER_PX_STAGE + BWD_FLOPS_PER_PX_STAGE)
        self.flops_per_px_stage = FLOPS_PER_PX_STAGE + BWD_FLOPS_PER_PX_STAGE
        adj = "bwd_adj" if bwd_algo == "fused" else f"tc_bwd_adj[{bwd_algo}]"
        dk = f"tc_bwd_dk[{bwd_algo}]" if bwd_algo == "tf32" else "bwd_dk"
        self.kernel = (B.tnrd_forward_kernel(self.m.params(), n, S, S, B.ALGO[algo]) +
                       f" + bwd_prep/bwd_zb/{adj}/{dk}/bwd_reduce <7,48>")
        if algo != "fused":
            # the forward's filter bank and adjoint on the tensor cores, the rest FP32
            self.tensor_dtype = algo
            self.dtype = ("f32 (forward: split TF32 tensor-core products)" if algo == "tf32x3" else
                          f"{algo} operands, f32 accumulate (forward filter bank and adjoint); f32")
            self.conv_flops_per_px_stage = CONV_FLOPS_PER_PX_STAGE
            self.alu_flops_per_px_stage = ALU_FLOPS_PER_PX_STAGE + BWD_FLOPS_PER_PX_STAGE
        self.h2d = int((self.f_host.numel() + self.c_host.numel()) * 4)
        self.d2h = int(self.g_host.numel() * 4)
        fwd = {"fused": "", "tf32": ", TF32 tensor-core forward",
               "bf16": ", BF16 tensor-core forward",
               "tf32x3": ", split-TF32 tensor-core forward"}[algo]
        fwd += {"fused": (", FP32 backward" if algo != "fused" else ""),
                "tf32x3": ", backward adjoint on split-TF32 tensor cores",
                "tf32": ", backward adjoint and filter gradient on TF32 tensor cores"}[bwd_algo]
        self.config = {"workload": f"TRDMD training step (forward + backward), {n} crops of "
                                   f"{S}x{S}, L=1, 7x7x48, 63 RBF, T={T_}, loss 1/2|u_T - clean|^2, "
                                   "gradients of all filters, RBF weights and lambda" + fwd,
                       "batch": n, "crop": S, "ksize": KS, "nfilt": NK, "nrbf": 63, "T": T_,
                       "l2": f"working set (checkpoints + response planes, "
                             f"{self.ws_bytes / 2 ** 20:.0f} MiB workspace) larger than L2"}

    def step(self):
        from paper_1702_07482_gb300 import ops
        u = ops.forward(self.m, self.f_dev, keep_stages=True, algo=self.algo, out=self.u_all,
                        W=self.S)
        e = u[-1] - self.c_dev
        self.grads = ops.backward(self.m, self.f_dev, u, e, want_grad_u0=False, W=self.S,
                                  workspace=self.ws, algo=self.bwd_algo)

    def e2e(self):
        import torch
        self.f_dev.copy_(self.f_host, non_blocking=True)
        self.c_dev.copy_(self.c_host, non_blocking=True)
        self.step()
        _, gk, gw, gl = self.grads
        flat = torch.cat([gk.reshape(-1), gw.reshape(-1), gl.reshape(-1)])
        self.g_host.copy_(flat, non_blocking=True)

    def accuracy(self):
        """Gradients of crop 0 alone (the step's kernels on a batch of one)
        against the FP64 oracle's: relative L2 error of each group (the filters
        and the RBF weights of each stage, lambda), the largest reported."""
        import numpy as np
        import torch
        import oracle
        from paper_1702_07482_gb300 import ops
        f0 = self.f_dev[:1]
        u = ops.forward(self.m, f0, keep_stages=True, algo=self.algo, W=self.S)
        _, gk, gw, gl = ops.backward(self.m, f0, u, (u[-1] - self.c_dev[:1]).contiguous(),
                                     want_grad_u0=False, W=self.S, algo=self.bwd_algo)
        torch.cuda.synchronize()
        oracle.build()
        fo = self.f[0].astype(np.float64)
        t0 = time.perf_counter()
        ua = oracle.forward(fo, self.p)
        _, rk, rw, rl = oracle.backward(fo, self.p, ua, ua[-1] - self.clean[0].astype(np.float64))
        self._full = (self.S * self.S, time.perf_counter() - t0)
        rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))
        c = lambda t: t.double().cpu().numpy()
        gk, gw, gl = c(gk), c(gw), c(gl)
        errs = {"lambda": rel(gl, rl)}
        for t in range(self.T):
            errs[f"filters_{t}"] = rel(gk[t], rk[t])
            errs[f"rbf_w_{t}"] = rel(gw[t], rw[t])
        worst = max(errs, key=errs.get)
        return {"vs": "FP64 oracle", "image": f"crop 0 ({self.S}x{self.S}) as a batch of one",
                "grad_rel_l2_max": errs[worst], "worst_group": worst,
                "grad_rel_l2": errs}

    def cpu_baseline(self):
        import oracle
        oracle.build()
        f0 = self.f[0].astype("float64")
        c0 = self.clean[0].astype("float64")

        def band(r):
            ua = oracle.forward(f0[:r].copy(), self.p)
            oracle.backward(f0[:r].copy(), self.p, ua, ua[-1] - c0[:r])

        r = _oracle_baseline(band, 6, self.S, self.S, f"crop 0 ({self.S}x{self.S})",
                             getattr(self, "_full", None))
        r["sample"] = r["sample"].replace("all stages", "forward + backward of all stages")
        r["sample_1thread"] = r["sample_1thread"].replace("all stages",
                                                          "forward + backward of all stages")
        return r


class Fit(Train):
    """One Adam iteration of joint training (Sec. 3.2) on the training-step
    batch: forward, backward, zero-mean filter projection and the update of
    filters, RBF weights and beta = log lambda.  With N GPUs every rank trains
    on its own 32 crops and the gradients are summed over the ranks (one
    all-reduce per step): weak scaling."""

    def __init__(self, dev, algo="fused"):
        super().__init__(dev, algo=algo)
        import torch
        from paper_1702_07482_gb300 import train
        self.tp = train.Params.from_model(self.p.filters, self.p.rbf_w, self.p.lam, device=dev)
        self.opt = torch.optim.Adam(self.tp.tensors(), lr=1e-3)
        self.f_img = self.f_dev[..., :self.S]
        self.c_img = self.c_dev[..., :self.S]
        self.loss_host = torch.empty(1, dtype=torch.float32).pin_memory()
        self.d2h = 4
        self.kernel = self.kernel + " + torch Adam on the parameters"
        self.config = dict(self.config)
        self.config["workload"] = (f"TRDMD joint training iteration (Adam, lr 1e-3): forward + "
                                   f"backward + update, {self.n} crops of {self.S}x{self.S}, L=1, "
                                   f"7x7x48, 63 RBF, T={self.T}, loss 1/2|u_T - clean|^2")

    def step(self):
        from paper_1702_07482_gb300 import train
        from paper_1702_07482_gb300.shard import allreduce_gradients
        self.opt.zero_grad(set_to_none=False)
        self.loss = train.loss_sum(train.cascade(self.tp, self.f_img, algo=self.algo),
                                   self.c_img)
        self.loss.backward()
        allreduce_gradients(self.tp.tensors())   # data-parallel ranks (no-op on one GPU)
        self.opt.step()

    def e2e(self):
        self.f_dev.copy_(self.f_host, non_blocking=True)
        self.c_dev.copy_(self.c_host, non_blocking=True)
        self.step()
        self.loss_host.copy_(self.loss.detach().reshape(1), non_blocking=True)


class Quality(Workload):
    """Quality indexes of Sec. 4 (PSNR, MSSIM, EC, RI_M, RI_V, C) of 16 images of
    2048 x 2048 (reference, despeckled-like result, L = 2 speckled input)."""

    def __init__(self, dev, n=16, S=2048, cfg=5):
        super().__init__(dev)
        import numpy as np
        import torch
        import synth
        from paper_1702_07482_gb300 import binding as B
        self.n, self.S = n, S
        hosts = [torch.empty((n, S, S), dtype=torch.float32).pin_memory() for _ in range(3)]
        g = np.random.Generator(np.random.PCG64(synth.seed_for(cfg, 0, "params") + 9))
        for i in range(n):
            clean, f = synth.single_image(S, S, 2, cfg, index=i)
            img = np.maximum(clean * (1.0 + 0.05 * g.standard_normal(clean.shape)), 0.5)
            hosts[0][i] = torch.from_numpy(clean.astype(np.float32))
            hosts[1][i] = torch.from_numpy(img.astype(np.float32))
            hosts[2][i] = torch.from_numpy(f.astype(np.float32))
            if i == 0:
                self.sample = [h[0].numpy().astype(np.float64) for h in hosts]
        self.hosts = hosts
        self.devs = [h.to(dev) for h in hosts]
        self.out = torch.empty((n, B.QUALITY_COUNT), dtype=torch.float64, device=dev)
        self.out_host = torch.empty_like(self.out, device="cpu").pin_memory()
        self.ws_bytes = B.tnrd_quality_workspace_size(n, S, S)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        self.sp = torch.cuda.current_stream(dev).cuda_stream
        self.px = n * S * S
        self.launches = 2
        # ALU-bound: ~1622 flops for 12 bytes (reference, result, noisy) per pixel
        self.flops = float(self.px) * QUALITY_FLOPS_PER_PX
        self.flops_per_px_stage = QUALITY_FLOPS_PER_PX
        self.kernel = "quality_partials + quality_finish"
        self.h2d = int(3 * n * S * S * 4)
        self.d2h = int(self.out.numel() * 8)
        self.config = {"workload": f"quality indexes of Sec. 4 (PSNR, MSSIM 11x11 Gaussian, "
                                   f"Laplacian edge correlation, ratio-image mean/variance, "
                                   f"coefficient of variation), {n} x {S}x{S}",
                       "images": n, "H": S, "W": S,
                       "l2": f"inputs ({self.h2d / 2 ** 20:.0f} MiB) larger than L2"}

    def step(self):
        from paper_1702_07482_gb300 import binding as B
        B.tnrd_quality(self.devs[0], self.devs[1], self.devs[2], self.n, self.S, self.S, self.S,
                       255.0, self.out, self.ws, self.ws_bytes, self.sp)

    def e2e(self):
        for d, h in zip(self.devs, self.hosts):
            d.copy_(h, non_blocking=True)
        self.step()
        self.out_host.copy_(self.out, non_blocking=True)

    def cpu_baseline(self):
        from oracle import quality as Q
        r = 256
        t0 = time.perf_counter()
        Q.indexes(*(a[:r, :r] for a in self.sample))
        dt = time.perf_counter() - t0
        return {"value": r * r / dt / 1e6, "unit": "Mpixel/s", "cores": 1, "kind": "oracle",
                "sample": f"all six indexes of a {r}x{r} crop of image 0 ({dt:.1f} s, numpy, "
                          f"one thread)", "cpu_model": _cpu_model(), "nproc": os.cpu_count()}


class Mixed(Workload):
    """16 images of 2048 x 2048, L = 2, 7x7x48, T = 8, as one batch."""

    def __init__(self, dev, algo="tf32", n=16, S=2048, T_=8, cfg=5):
        super().__init__(dev)
        import numpy as np
        import torch
        import synth
        from paper_1702_07482_gb300 import binding as B
        from paper_1702_07482_gb300 import ops
        self.T, self.n, self.S, self.algo = T_, n, S, algo
        self.tensor_dtype = algo if algo in TENSOR_RATIO else None
        self.dtype = {"tf32": "tf32 operands, f32 accumulate",
                      "bf16": "bf16 operands, f32 accumulate",
                      "tf32x3": "f32 (split TF32 tensor-core products)"}.get(algo, "f32")
        self.p = _p32(synth.params(T_, KS, NK, seed=synth.seed_for(cfg, 0, "params")))
        self.m = ops.Model.create(self.p.filters, self.p.rbf_w, self.p.lam, device=dev)
        self.prm = self.m.params()
        self.f_host = torch.empty((n, S, S), dtype=torch.float32).pin_memory()
        self.f0 = None
        for i in range(n):
            _, f = synth.single_image(S, S, 2, cfg, index=i)
            self.f_host[i] = torch.from_numpy(f.astype(np.float32))
            if i == 0:
                self.f0 = f.astype(np.float32).astype(np.float64)
        self.f_dev = self.f_host.to(dev)
        self.u_dev = torch.empty_like(self.f_dev)
        self.u_host = torch.empty_like(self.f_host).pin_memory()
        self.code = B.ALGO["fused" if algo == "fp32" else algo]
        self.ws_bytes = B.tnrd_workspace_size(B.OP_FORWARD, self.prm, n, S, S, S, 0, self.code)
        self.ws = torch.empty(max(self.ws_bytes, 1), dtype=torch.uint8, device=dev)
        self.sp = torch.cuda.current_stream(dev).cuda_stream
        self.px = n * S * S
        self.launches = T_
        self.flops = float(self.px) * T_ * FLOPS_PER_PX_STAGE
        self.flops_per_px_stage = FLOPS_PER_PX_STAGE
        self.kernel = B.tnrd_forward_kernel(self.prm, n, S, S, self.code) + \
            {"tf32": " (tcgen05 TF32 filter bank and adjoint, FP32 phi/prox)",
             "bf16": " (tcgen05 BF16 filter bank and adjoint, FP32 phi/prox)",
             "tf32x3": " (tcgen05 split-TF32 filter bank and adjoint, FP32 phi/prox)"}.get(
                algo, " (FP32)")
        prec = (f"filter bank and adjoint on tensor cores ({PREC_TEXT[algo]}), phi and prox FP32"
                if algo in PREC_TEXT else "plain FP32 fused stage kernel")
        self.h2d = self.d2h = int(self.f_host.numel() * 4)
        self.config = {"workload": f"TRDMD forward, {n} x {S}x{S}, L=2, 7x7x48, 63 RBF, T={T_}, "
                                   f"{prec}",
                       "images": n, "H": S, "W": S, "ksize": KS, "nfilt": NK, "nrbf": 63, "T": T_,
                       "looks": 2, "precision": algo,
                       "l2": f"inputs ({self.h2d / 2 ** 20:.0f} MiB) larger than L2"}

    def step(self):
        from paper_1702_07482_gb300 import binding as B
        B.tnrd_forward(self.prm, self.n, self.S, self.S, self.S, self.f_dev, self.u_dev, 0,
                       self.code, self.ws, self.ws_bytes, self.sp)

    def e2e(self):
        self.f_dev.copy_(self.f_host, non_blocking=True)
        self.step()
        self.u_host.copy_(self.u_dev, non_blocking=True)

    def accuracy(self):
        """u_T of a whole 1024 x 1024 image (the top-left crop of image 0, run as
        its own image through the same kernel) against the FP64 oracle."""
        import torch
        from paper_1702_07482_gb300 import binding as B
        S = 1024
        f = self.f0[:S, :S].copy()
        fd = torch.tensor(f, dtype=torch.float32, device=self.dev).unsqueeze(0).contiguous()
        ud = torch.empty_like(fd)
        nb = B.tnrd_workspace_size(B.OP_FORWARD, self.prm, 1, S, S, S, 0, self.code)
        ws = torch.empty(max(nb, 1), dtype=torch.uint8, device=self.dev)
        B.tnrd_forward(self.prm, 1, S, S, S, fd, ud, 0, self.code, ws, nb, self.sp)
        torch.cuda.synchronize()
        got = ud[0].double().cpu().numpy()
        u, dt = _timed_oracle_forward(f, self.p)
        self._full = (S * S, dt)
        return _accuracy(got, u[-1], f"{S}x{S} top-left crop of image 0 run as its own image, "
                                     f"L=2, T={self.T} (u_T)")

    def cpu_baseline(self):
        import oracle
        band = lambda r: oracle.forward(self.f0[:r, :1024].copy(), self.p)
        return _oracle_baseline(band, 4, 1024, 1024, "the 1024x1024 crop of image 0",
                                getattr(self, "_full", None))


def make_workload(name, dev):
    if name == "fwd512":
        return Fwd(dev)
    if name == "fwd512_unfused":
        return Fwd(dev, algo="unfused")
    if name == "quality":
        return Quality(dev)
    if name == "fwd512_gauss":
        return Fwd(dev, data_term=1)
    if name == "fwd512_proj":
        return Fwd(dev, data_term=2)
    if name == "small128":
        return Fwd(dev, H=128, W=128, ks=5, nk=24, cfg=1)
    if name == "batched":
        return Batched(dev)
    if name == "batched_tf32":
        return Batched(dev, algo="tf32")
    if name == "batched_bf16":
        return Batched(dev, algo="bf16")
    if name == "batched_tf32x3":
        return Batched(dev, algo="tf32x3")
    if name == "train":
        return Train(dev)
    if name == "train_tf32":
        return Train(dev, algo="tf32")
    if name == "train_tf32x3":
        return Train(dev, algo="tf32x3", bwd_algo="tf32x3")
    if name == "train_tc":
        return Train(dev, algo="tf32", bwd_algo="tf32")
    if name == "fwd512_tf32x3":
        return Fwd(dev, algo="tf32x3")
    if name == "mixed_tf32x3":
        return Mixed(dev, algo="tf32x3")
    if name == "train_bf16":
        return Train(dev, algo="bf16")
    if name == "fit":
        return Fit(dev)
    if name == "fit_tf32":
        return Fit(dev, algo="tf32")
    if name == "mixed_tf32":
        return Mixed(dev, algo="tf32")
    if name == "mixed_bf16":
        return Mixed(dev, algo="bf16")
    if name == "mixed_fp32":
        return Mixed(dev, algo="fp32")
    raise ValueError(name)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    import synth
    oracle.build()
    p = _p32(synth.params(T, KS, NK, seed=synth.seed_for(CFG_ID, 0, "params")))
    _, f = synth.single_image(H, W, L, CFG_ID, index=0)
    f = f.astype(np.float32).astype(np.float64)
    band = lambda r: oracle.forward(f[:r].copy(), p)
    rows, _ = _rows_rate(band, 8, 2.0, H)     # one step about 1-4 s
    for _ in range(args.warmup):
        band(rows)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        band(rows)
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
                         "sample": sample, "cpu_model": _cpu_model(), "nproc": os.cpu_count()},
        "e2e": {"value": value, "unit": "Mpixel/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# Per pixel-stage at 7x7x48: the filter bank and the adjoint are the two
# contractions (2 x 2 N_k k^2 flops), phi and the prox the rest.
CONV_FLOPS_PER_PX_STAGE = 2 * 2 * NK * KS * KS
ALU_FLOPS_PER_PX_STAGE = 2 * NK * 63 + 12
# dense tensor-core rates relative to BF16 (nominal: TF32 1.1, BF16 2.25 PFLOP/s);
# split TF32 spends three TF32 products on each product of the algorithm
TENSOR_RATIO = {"tf32": 1.1 / 2.25, "bf16": 1.0, "tf32x3": 1.1 / 2.25 / 3}
PREC_TEXT = {"tf32": "TF32 operands, FP32 accumulate",
             "bf16": "BF16 operands, FP32 accumulate",
             "tf32x3": "split TF32 operands (hi + lo, three products), FP32 accumulate"}


def _split_roofline(wl, tc, ms, peaks, src, peak_fp32, n_sm, sm_max):
    """Roofline of a tensor-core stage: the step cannot be shorter than
    T_min = max(conv flops / tensor peak, (phi + prox) flops / FP32 peak); the
    binding term is reported (frac = T_min / T)."""
    px_st = wl.flops / wl.flops_per_px_stage
    conv = px_st * getattr(wl, "conv_flops_per_px_stage", CONV_FLOPS_PER_PX_STAGE)
    alu = px_st * getattr(wl, "alu_flops_per_px_stage", ALU_FLOPS_PER_PX_STAGE)
    bf = float(peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops") or 1700.0)
    tpeak = bf * TENSOR_RATIO[tc]
    t = ms / 1e3
    terms = {
        "tensor": {"flops": conv, "achieved": conv / t / 1e12, "peak": tpeak,
                   "frac": conv / t / 1e12 / tpeak,
                   "peak_source": f"{src} bf16_tflops_sustained {bf:.1f} x nominal {tc}/bf16 "
                                  f"ratio {TENSOR_RATIO[tc]:.3f}" +
                               (" (TF32 / 3: three TF32 products per product)" if tc == "tf32x3"
                                else "")},
        "alu": {"flops": alu, "achieved": alu / t / 1e12, "peak": peak_fp32,
                "frac": alu / t / 1e12 / peak_fp32,
                "peak_source": f"derived: {n_sm} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz"},
    }
    bound = max(terms, key=lambda k: terms[k]["flops"] / terms[k]["peak"])
    b = terms[bound]
    return {"bound": bound, "achieved": b["achieved"], "peak": b["peak"], "unit": "TFLOP/s",
            "frac": b["frac"], "traffic": wl.traffic, "kernel": wl.kernel,
            "launches_per_step": wl.launches,
            "achieved_basis": "split roofline: T_min = max(filter bank + adjoint flops / tensor "
                              "peak, (phi + prox" + (" + FP32 backward" if hasattr(
                                  wl, "alu_flops_per_px_stage") else "") +
                              ") flops / FP32 peak); frac = T_min / step time "
                              "of the binding term",
            "terms": terms, "peak_source": b["peak_source"]}


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and args.workload not in ("fwd512", "fit", "fit_tf32"):
        if rank == 0:
            print(json.dumps({"workload": args.workload,
                              "unavailable": "multi-GPU runs use the fwd512 (independent images) "
                                             "or fit (data-parallel training) workloads"}))
        return 0
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1702_07482_gb300 import binding, build
    build.build()
    binding.load()
    wl = make_workload(args.workload, dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def timed(fn, clk):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        barrier()
        t0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(i & 0xFF)          # evict the previous step's data from L2
            evs[i][0].record(stream)
            fn()
            evs[i][1].record(stream)
        barrier()
        if hasattr(clk, "mark"):
            clk.mark(t0, time.perf_counter())
        return [a.elapsed_time(b) for a, b in evs]

    for _ in range(max(args.warmup, 3)):
        flush.fill_(0)                     # its first launch loads the fill kernel: not in the window
        wl.step()
    barrier()
    sampler = NvmlClocks(dev)
    if not sampler.ok:
        sampler = ClockSampler(local)
    sampler.start()
    if not hasattr(sampler, "mark"):
        time.sleep(0.3)   # nvidia-smi needs a moment before its first sample
    step_ms = timed(wl.step, sampler)
    # end to end through the C ABI: pinned host inputs -> device -> path ->
    # pinned host result, all inside the events
    for _ in range(3):
        wl.e2e()
    e2e_ms = timed(wl.e2e, sampler)
    # the default workload also on the split-TF32 tensor-core stage (FP32
    # accuracy on the tensor cores), reported beside the headline, not as it
    alt_wl = alt_ms = None
    if args.workload == "fwd512" and world == 1 and not args.no_alt:
        alt_wl = Fwd(dev, algo="tf32x3")
        for _ in range(max(args.warmup, 3)):
            alt_wl.step()
        barrier()
        alt_ms = timed(alt_wl.step, sampler)
    clocks = sampler.stop()

    from paper_1702_07482_gb300.shard import global_rate
    value, ms = global_rate(wl.px, statistics.mean(step_ms))
    e2e_value, ms_e2e = global_rate(wl.px, statistics.mean(e2e_ms))
    out = None
    if rank == 0:
        peaks, src = _peaks()
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        sm_max = float(peaks.get("sm_max_mhz", 2070.0))
        peak_tf = _fp32_peak_tflops(sm_max, n_sm)
        achieved_tf = wl.flops / (ms / 1e3) / 1e12
        # accuracy first: its whole-image oracle run is the all-core CPU sample
        acc = wl.accuracy() if (hasattr(wl, "accuracy") and not args.no_accuracy) else None
        cpu = None if args.no_cpu_baseline else wl.cpu_baseline()
        out = {
            "metric": METRIC, "value": value, "unit": "Mpixel/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": getattr(wl, "dtype", "f32"), "data": "synthetic",
            "config": wl.config,
            "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": peak_tf,
                          "unit": "TFLOP/s", "frac": achieved_tf / peak_tf,
                          "traffic": wl.traffic,
                          "kernel": wl.kernel,
                          "launches_per_step": wl.launches,
                          "achieved_basis": "algorithmic flops per step / step time (the "
                                            "step's launches run back to back on one stream)",
                          "peak_source": f"derived: {n_sm} SMs x 128 FP32 lanes x 2 x "
                                         f"{sm_max:.0f} MHz ({src} sm_max_mhz)",
                          "flops_per_px_stage": wl.flops_per_px_stage},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "Mpixel/s", "h2d_bytes_per_step": wl.h2d,
                    "d2h_bytes_per_step": wl.d2h},
            "gpu_launches": args.steps * wl.launches,
            "clocks": clocks,
        }
        if acc is not None:
            out["accuracy"] = acc
        tc = getattr(wl, "tensor_dtype", None)
        if tc:
            out["roofline"] = _split_roofline(wl, tc, ms, peaks, src, peak_tf, n_sm, sm_max)
        if alt_ms:
            a_ms = statistics.mean(alt_ms)
            alt = {"what": "the same workload and inputs on the split-TF32 tensor-core stage "
                           "(TNRD_ALGO_TC_TF32X3: operands as TF32 high part + TF32 remainder, "
                           "three products, FP32 accumulation); reported beside the headline",
                   "value": alt_wl.px / (a_ms / 1e3) / 1e6, "unit": "Mpixel/s", "ms_per_step": a_ms,
                   "steps": args.steps, "kernel": alt_wl.kernel, "dtype": alt_wl.dtype,
                   "gpu_launches": args.steps * alt_wl.launches,
                   "roofline": _split_roofline(alt_wl, "tf32x3", a_ms, peaks, src, peak_tf, n_sm,
                                               sm_max)}
            if getattr(wl, "ref_uT", None) is not None:
                alt_wl.step()
                torch.cuda.synchronize(dev)
                got = alt_wl.u_dev[0, :, :alt_wl.Ww].double().cpu().numpy()
                alt["accuracy"] = _accuracy(got, wl.ref_uT, f"{alt_wl.Hh}x{alt_wl.Ww} image (u_T)")
            out["fp32_accurate_tensor_core"] = alt
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
    ap.add_argument("--no-alt", action="store_true",
                    help="fwd512: skip the split-TF32 measurement reported beside the headline")
    ap.add_argument("--workload", default="fwd512",
                    choices=["fwd512", "fwd512_unfused", "small128", "batched", "batched_tf32",
                             "batched_bf16", "batched_tf32x3", "train", "train_tf32", "train_bf16",
                             "train_tf32x3",
                             "train_tc", "fwd512_tf32x3", "mixed_tf32x3",
                             "fit", "fit_tf32", "fwd512_gauss", "fwd512_proj", "quality", "mixed_tf32",
                             "mixed_bf16", "mixed_fp32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the whole-image comparison with the FP64 oracle")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
