#!/usr/bin/env python
"""Benchmark: ensemble Power Doppler delay-and-sum, points per second (Eq. 1).

Workload: the rotating-disk Doppler benchmark shape of Sec. 4.1 as a seeded synthetic
stand-in -- 256 x 256 pixels at 0.1 mm, 128-element linear array, one 0-degree plane
wave, 32 frames, 2048 complex64 samples per channel, F# 1.0 -- writing both the complex
frames (B-mode) and Power Doppler.  One step = one mach_power_doppler call on IQ already
resident in HBM; L2 is flushed (256 MB write, then 256 MB read) between steps, outside the timed events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: each rank beamforms its own acquisition (weak scaling, no
data-path collective); the time is the maximum over ranks.  ``--impl reference`` times
the FP64 CPU oracle on the same workload instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DAS points/s (voxel x channel x transmit x frame, Eq. 1)"
UNIT = "points/s"
PAPER_POINTS_PER_S = 258_052_096 / 0.23e-3      # Sec. 4.2: 0.23 ms on an RTX 5090, 251^2 px
KERNEL_SOURCES = ("k_das.cu", "k_das_staged.cu", "k_das_exact.cu", "das_staged.cuh", "k_das_table.cu", "das_term.cuh", "tap_mac.cuh",
                  "async_copy.cuh", "mach_internal.h")
FLUSH_BYTES = 256 << 20                           # > 129 MB L2


class L2Flush:
    """Evicts L2 between timed steps: writes a buffer larger than L2, then reads a second
    one, so that a timed kernel starts with L2 holding neither its inputs nor dirty lines
    whose write-back it would be charged for.  `zero_()` runs both, outside the events."""

    def __init__(self, device="cuda"):
        import torch
        self.w = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=device)
        self.r = torch.ones(FLUSH_BYTES // 4, dtype=torch.float32, device=device)

    def zero_(self):
        self.w.zero_()
        self.r.sum()



def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="doppler2d")
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variant", default="", help="force a kernel variant (ablations)")
    ap.add_argument("--term-table", action="store_true",
                    help="time the plan that stores every term (mach_das_desc.term_table) instead of the "
                         "on-the-fly delays")
    ap.add_argument("--ragged-n", type=int, default=64, help="instances of the ragged batch")
    ap.add_argument("--ragged-scale", type=float, default=1.0, help="grid scale of the ragged batch")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--iq-dtype", default="c64split", choices=["c64", "f16x2", "bf16x2", "c64split"],
                    help="IQ storage the timed kernel reads (prepared by K0 outside the timed region)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other workloads (volume3d, bmode2d, ragged batch, learned compounding) "
                         "reported beside the headline")
    ap.add_argument("--sweep-axes", default="voxels,channels,frames", help="axes of --workload sweep")
    return ap.parse_args()


# ---------------------------------------------------------------- helpers ----

def dist_init(n):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and not dist.is_initialized():
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return rank, world, local


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2604_06257_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_entry(variant: str, workload: str) -> dict:
    """The committed ncu figures of one launch (DRAM bytes, L2 bytes and the L2 peak
    sector rate), if they were taken on the current kernel sources; else {}."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        data = json.load(open(path))
    except (OSError, ValueError):
        return {}
    e = data.get(f"{variant}@{workload}")
    if not e or e.get("kernel_sha") != kernel_hash():
        return {}
    return e


def profiled_traffic(variant: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, or None."""
    return profiled_entry(variant, workload).get("dram_bytes_per_launch")


class Clocks:
    """SM clock, its maximum, power and clock-event (throttle) reasons of this process's
    GPU, sampled DURING the timed region.

    NVML (the library nvidia-smi reads) is polled from a background thread every ~2 ms,
    so that even a region of a few milliseconds gets samples; ``nvidia-smi -lms 200`` is
    the fallback when NVML cannot be loaded.  Only settings are read, nothing is set."""
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
    # nvmlClocksEventReason* bits (public NVML API)
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}
    Q = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str):
        self.uuid = uuid.replace("GPU-", "").lower()
        self.samples = []
        self.proc = None
        self.thread = None
        self.nvml = None
        self.dev = None
        try:
            import ctypes
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() == 0:
                h = ctypes.c_void_p()
                if nv.nvmlDeviceGetHandleByUUID(("GPU-" + self.uuid).encode(), ctypes.byref(h)) == 0:
                    self.nvml, self.dev = nv, h
        except OSError:
            self.nvml = None

    def _poll(self):
        import ctypes
        nv, h = self.nvml, self.dev
        sm, mx, pw, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        get_reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            nv.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self._stop:
            ok = nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(sm)) == 0     # NVML_CLOCK_SM
            ok = ok and nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0
            p_ok = nv.nvmlDeviceGetPowerUsage(h, ctypes.byref(pw)) == 0
            r_ok = get_reasons(h, ctypes.byref(rs)) == 0
            if ok:
                self.samples.append((time.perf_counter(), float(sm.value), float(mx.value),
                                     pw.value / 1e3 if p_ok else None, int(rs.value) if r_ok else 0))
            time.sleep(0.002)

    def start(self):
        self._stop = False
        if self.nvml is not None:
            import threading
            self.thread = threading.Thread(target=self._poll, daemon=True)
            self.thread.start()
            return
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self, t_begin=None, t_end=None):
        """Summary of the samples taken between t_begin and t_end (perf_counter times;
        all samples when not given)."""
        if self.thread is not None:
            self._stop = True
            self.thread.join()
            rows = [r for r in self.samples if (t_begin is None or r[0] >= t_begin) and (t_end is None or r[0] <= t_end)]
            if not rows:
                return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0, "source": "nvml"}
            pw = [r[3] for r in rows if r[3] is not None]
            reasons = sorted({n for r in rows for n, b in self.BITS.items() if r[4] & b})
            return {"sm_mhz": statistics.median(r[1] for r in rows), "sm_max_mhz": max(r[2] for r in rows),
                    "power_w_median": statistics.median(pw) if pw else None, "reasons": reasons,
                    "samples": len(rows), "source": "NVML, polled every ~2 ms during the timed region"}
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.flush()
        rows = []
        for line in open(self.out.name):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9 or not parts[0].lower().endswith(self.uuid[-12:]):
                continue
            rows.append(parts)
        os.unlink(self.out.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        pw = [float(r[3]) for r in rows if r[3].replace(".", "", 1).isdigit()]
        reasons = sorted({n for r in rows for n, v in zip(self.NAMES, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_median": statistics.median(pw) if pw else None,
                "reasons": reasons, "samples": len(rows), "source": "nvidia-smi -lms 200"}


DESCRIBE = {"doppler2d": "rotating-disk Doppler stand-in (Sec. 4.1 shape)",
            "ulm3d": "3D ULM shape (Sec. 6: 94x94x178 voxels, 1024 el, 5 angles)",
            "volume3d": "32x32 matrix-array volume (Sec. 6 shape)",
            "bmode2d": "steered plane-wave B-mode (Sec. 2.1 compounding)"}


def workload_config(acq, extra=None):
    kind = acq.name.split("_")[0]
    grid = "x".join(str(n) for n in acq.grid_dims if n > 1)
    d = {"workload": f"{acq.name}: {DESCRIBE.get(kind, kind)}, {grid} voxels, {acq.n_elem} ch, "
                     f"{acq.n_tx} tx, {acq.n_frames} frames, {acq.n_samples} samples, {acq.iq_dtype} IQ, "
                     f"F# {acq.f_number} {acq.apod}; outputs complex frames + Power Doppler",
         "voxels": acq.n_vox, "channels": acq.n_elem, "transmits": acq.n_tx,
         "frames": acq.n_frames, "samples": acq.n_samples,
         "points_per_step": acq.points,
         "l2": "flushed between timed steps (256 MB write, then 256 MB read, outside the timed events)"}
    if extra:
        d.update(extra)
    return d


def oracle_sample(acq, iq_host, seconds, min_vox=64):
    """Time the oracle on a bounded sample of the workload: the whole workload repeated
    until about ``seconds`` of work if one pass is shorter, else an evenly strided voxel
    subset sized to about ``seconds``."""
    import numpy as np
    import oracle
    cal = np.arange(0, acq.n_vox, max(1, acq.n_vox // 512))[:512]
    t = time.perf_counter()
    oracle.das(acq, iq_host, cal, want_y=False)
    dt = max(time.perf_counter() - t, 1e-6)
    full_est = dt * acq.n_vox / len(cal)
    if full_est < seconds:
        reps, done, t0 = 0, 0.0, time.perf_counter()
        while done < seconds:
            oracle.das(acq, iq_host, None, want_y=True)
            reps += 1
            done = time.perf_counter() - t0
        pts = acq.points * reps
        sample = (f"the whole workload ({acq.n_vox} voxels, all channels, transmits and frames), "
                  f"{reps} passes in {done:.1f} s, FP64")
        return {"value": pts / done, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                "sample": sample}
    n = int(min(acq.n_vox, max(min_vox, len(cal) * seconds / dt)))
    idx = np.linspace(0, acq.n_vox - 1, n).astype(np.int64)
    t = time.perf_counter()
    oracle.das(acq, iq_host, idx, want_y=True)
    dt = time.perf_counter() - t
    pts = n * acq.n_elem * acq.n_tx * acq.n_frames
    return {"value": pts / dt, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{n} of {acq.n_vox} voxels (evenly strided), all channels, transmits "
                      f"and frames; one pass, {dt:.2f} s, FP64"}


def count_active_terms(plan, V, C, T, chunk_terms=1 << 26):
    """Terms (voxel, element, transmit) inside the aperture and the sample range, as the
    kernels evaluate them (mach_das_terms, indices only, in voxel chunks)."""
    import torch
    import paper_2604_06257_gb300 as m
    per = max(1, chunk_terms // (C * T))
    i0 = torch.empty(min(per, V) * C * T, dtype=torch.int32, device="cuda")
    total = 0
    for a in range(0, V, per):
        n = min(per, V - a)
        idx = torch.arange(a, a + n, dtype=torch.int64, device="cuda")
        m.mach_das_terms(plan.handle, idx, i0=i0[: n * C * T])
        total += int((i0[: n * C * T] >= 0).sum().item())
    return total


def active_fraction_sampled(plan, acq, n=2048, seed=0):
    """Share of terms (voxel, element, transmit) inside the aperture and the sample range,
    estimated on n evenly spread voxels (mach_das_terms, indices only)."""
    import numpy as np
    import torch
    import paper_2604_06257_gb300 as m
    V, C, T = acq.n_vox, acq.n_elem, acq.n_tx
    n = min(n, V)
    idx = torch.as_tensor(np.linspace(0, V - 1, n).astype(np.int64), device="cuda")
    i0 = torch.empty(n * C * T, dtype=torch.int32, device="cuda")
    m.mach_das_terms(plan.handle, idx, i0=i0)
    return float((i0 >= 0).sum().item()) / (n * C * T)


def time_plan(plan, iq, pd, y, steps, warmup, flush, stream):
    """Mean device time of one mach_power_doppler call (CUDA events on the launching
    stream, L2 flushed before every call, outside the events)."""
    import torch
    import paper_2604_06257_gb300 as m
    for _ in range(warmup):
        flush.zero_()
        m.mach_power_doppler(plan.handle, iq, pd, y)
    evs = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        m.mach_power_doppler(plan.handle, iq, pd, y)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    return statistics.mean(a.elapsed_time(b) for a, b in evs) / 1e3


def peaks_and_units():
    import torch
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = props.multi_processor_count
    return {"n_sm": n_sm, "sm_max": sm_max, "fp32_tflops": n_sm * 128 * 2 * sm_max * 1e6 / 1e12,
            "lds_gbs": n_sm * 128 * sm_max * 1e6 / 1e9, "hbm_gbs": float(peaks.get("hbm_gbs", 6800.0))}


def oracle_error(acq, iq_c64, y, pd, n_vox, iq_ref=None):
    """Part of the CPU baseline leg: NRMSE (dB) of the GPU frames and Power Doppler against
    the oracle on n_vox evenly spread voxels, with the plan's float32 delay contract and
    with exact (all-FP64) delays."""
    import numpy as np
    import torch
    import oracle
    V = acq.n_vox
    idx = np.unique(np.linspace(0, V - 1, n_vox).astype(np.int64))
    sel = torch.as_tensor(idx, device=y.device)
    ys, ps = y[sel].cpu().numpy().astype(np.complex128), pd[sel].cpu().numpy().astype(np.float64)
    ref = iq_c64.cpu() if iq_ref is None else iq_ref
    err = {"voxels": len(idx)}
    for mode in ("contract", "exact"):
        yr, pr = oracle.das(acq.replace(iq_dtype="c64"), ref, idx, mode=mode)
        err[mode] = {"frames_db": float(20 * np.log10(np.linalg.norm(ys - yr) / np.linalg.norm(yr))),
                     "pd_db": float(20 * np.log10(np.linalg.norm(ps - pr) / np.linalg.norm(pr)))}
    return err


def das_leg(acq, iq_c64, dt, steps, warmup, flush, stream, cpu_check=True, err_voxels=256):
    """One DAS + Power Doppler workload: points/s and roofline fractions; with the CPU
    baseline leg enabled, also the error of the timed output against the oracle."""
    import numpy as np
    import torch
    import synth
    import paper_2604_06257_gb300 as m
    a = acq.replace(iq_dtype=dt)
    x = synth.iqmod.to_storage(iq_c64, dt)
    V, F = a.n_vox, a.n_frames
    with m.Plan(**m.plan_kwargs(a)) as plan:
        info = plan.info()
        pd = torch.empty(V, dtype=torch.float32, device="cuda")
        y = torch.empty((V, F), dtype=torch.complex64, device="cuda")
        t = time_plan(plan, x, pd, y, steps, warmup, flush, stream)
        act = active_fraction_sampled(plan, a)
    pk = peaks_and_units()
    tf = act * a.n_elem * a.n_tx * V * F                      # active term-frames (estimated)
    bpt = 16 if dt in ("c64", "c64split") else 8
    out = {"value": a.points / t, "unit": UNIT, "ms_per_step": t * 1e3, "steps": steps, "warmup": warmup,
           "variant": info["variant"], "tile": info["tile"], "dtype": dt,
           "config": {"workload": a.name, "voxels": V, "channels": a.n_elem, "transmits": a.n_tx, "frames": F,
                      "samples": a.n_samples, "points_per_step": a.points},
           "roofline": {"bound": "alu", "unit": "TFLOP/s", "achieved": 16 * tf / t / 1e12, "peak": pk["fp32_tflops"],
                        "frac": 16 * tf / t / 1e12 / pk["fp32_tflops"],
                        "sm_load_path_frac": bpt * tf / t / 1e9 / pk["lds_gbs"],
                        "active_fraction": act, "active_fraction_source": "2048 evenly spread voxels"}}
    if cpu_check:
        ref = synth.iqmod.from_storage(x.cpu()) if dt in ("f16x2", "bf16x2") else None
        out["error_db_vs_oracle"] = oracle_error(a, iq_c64, y, pd, err_voxels, ref)
    return out


def ragged_leg(args, flush, steps=3):
    """The 64-instance ragged batch (float16 IQ) in one persistent launch replayed from a
    CUDA graph, default tile shapes."""
    import torch
    import synth
    from synth.ragged import ragged_instances
    import paper_2604_06257_gb300 as m
    acqs = ragged_instances(n=args.ragged_n, seed=4, iq_dtype="f16x2", scale=args.ragged_scale)
    kws = [m.plan_kwargs(a) for a in acqs]
    iqs, ys, pds = [], [], []
    for i, a in enumerate(acqs):
        iqs.append(synth.iqmod.to_f16x2(synth.random_iq(a, 1000 + i, device="cuda")))
        ys.append(torch.empty((a.n_vox, a.n_frames), dtype=torch.complex64, device="cuda"))
        pds.append(torch.empty(a.n_vox, dtype=torch.float32, device="cuda"))
    points = sum(a.points for a in acqs)
    with m.Batch(kws) as b:
        b.bind(iqs, ys, pds)
        b.run()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            b.run()
        for _ in range(2):
            g.replay()
        torch.cuda.synchronize()
        evs = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            evs.append((e0, e1))
        torch.cuda.synchronize()
        t = statistics.mean(a.elapsed_time(b_) for a, b_ in evs) / 1e3
        info = {k: v for k, v in b.info().items() if k != "shapes"}
    del iqs
    return {"value": points / t, "unit": UNIT, "ms_per_step": t * 1e3, "steps": steps,
            "config": {"workload": f"{len(acqs)} seeded instances (seed 4, 2D and 3D, 1-48 frames, 1-15 transmits, "
                                   "float16 IQ), one persistent launch replayed from a CUDA graph, default tile shapes",
                       "points_per_step": points}, "batch": info}


# ---------------------------------------------------------------- our arm ----

def run_ours(args):
    import numpy as np
    import torch
    import synth
    import paper_2604_06257_gb300 as m
    from paper_2604_06257_gb300 import build as pkg_build, counts, shard

    rank, world, local = dist_init(args.gpus)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU fallback)")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    pkg_build.build()
    m.lib()

    frames = synth.make_acquisition(args.workload, "full").n_frames
    if args.iq_dtype == "c64split" and (frames % 4 or frames <= 4):
        args.iq_dtype = "c64"          # split rows need a frame count that is a multiple of 4 above 4
    acq, iq = synth.make(args.workload, "full", device=dev, seed=synth.SEEDS[args.workload] + rank,
                         iq_dtype=args.iq_dtype)
    iq_c64 = iq                                     # complex64 [T, C, S, F]
    if args.iq_dtype != "c64":
        # K0 from the acquisition order [F, T, C, S] into the kernels' layout (untimed
        # preparation, as the paper excludes format conversion from its timing)
        iq = m.prepare_iq(iq_c64.permute(3, 0, 1, 2).contiguous(), "ftcs", args.iq_dtype)
    if args.variant:
        m.mach_debug_force_variant(args.variant)
    plan = m.Plan(**m.plan_kwargs(acq), term_table=args.term_table)
    m.mach_debug_force_variant(None)
    info = plan.info()
    V, F = acq.n_vox, acq.n_frames
    pd = torch.empty(V, dtype=torch.float32, device=dev)
    y = torch.empty((V, F), dtype=torch.complex64, device=dev)
    flush = L2Flush(dev)
    active_terms = count_active_terms(plan, V, acq.n_elem, acq.n_tx)
    active_points = active_terms * F
    launches_per_step = 1 + (1 if info["frame_tiles"] > 1 else 0)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        flush.zero_()
        m.mach_power_doppler(plan.handle, iq, pd, y)
    torch.cuda.synchronize()
    barrier()

    props = torch.cuda.get_device_properties(dev)
    clocks = Clocks(str(getattr(props, "uuid", "")))
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    torch.cuda.synchronize()
    barrier()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        m.mach_power_doppler(plan.handle, iq, pd, y)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    t_end = time.perf_counter()
    clk = clocks.stop(t_wall, t_end)
    t_wall = t_end - t_wall
    times_ms = [a.elapsed_time(b) for a, b in ev]
    t_sum = sum(times_ms) / 1e3
    t_max = shard.max_over_ranks(t_sum)
    value = world * acq.points * args.steps / t_max
    t_launch = statistics.mean(times_ms) / 1e3

    # roofline: the gather-MAC is bound by the SM load path and the FP32 pipe, not HBM.
    n_sm = props.multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    fp32_peak = n_sm * 128 * 2 * sm_max * 1e6 / 1e12                     # TFLOP/s
    flops = active_points * 16.0                                            # 8 FMA per term-frame
    achieved = flops / t_launch / 1e12
    comp = counts.compulsory_bytes(V, acq.n_elem, acq.n_tx, acq.n_samples, F, write_y=True, write_pd=True,
                                   iq_bytes=8 if args.iq_dtype in ("c64", "c64split") else 4)
    prof = profiled_entry(info["variant"] + ("+table" if args.term_table else ""), acq.name)
    traffic = prof.get("dram_bytes_per_launch")
    roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak, "traffic": traffic,
            "kernel": info["variant"],
            "peak_source": f"FP32 FMA: {n_sm} SMs x 128 lanes x 2 flop x {sm_max:.0f} MHz "
                           "(max SM clock, MEASURED_PEAKS.json)",
            "algorithmic": "16 flop (8 FP32 FMA) per active term-frame; active = in aperture "
                           f"and in range: {active_terms} of {V * acq.n_elem * acq.n_tx} terms",
            "hbm": {"compulsory_bytes": comp, "achieved_gbs": comp / t_launch / 1e9,
                    "peak_gbs": hbm_peak, "frac": comp / t_launch / 1e9 / hbm_peak},
            "sm_load_path": {"bytes_per_term_frame": 16 if args.iq_dtype in ("c64", "c64split") else 8,
                             "achieved_gbs": active_points * (16 if args.iq_dtype in ("c64", "c64split") else 8)
                             / t_launch / 1e9,
                             "peak_gbs": n_sm * 128 * sm_max * 1e6 / 1e9,
                             "peak_source": f"shared-memory load path: {n_sm} SMs x 128 B/clk x {sm_max:.0f} MHz",
                             "frac": active_points * (16 if args.iq_dtype in ("c64", "c64split") else 8)
                             / t_launch / (n_sm * 128 * sm_max * 1e6)}}
    if prof.get("l2_bytes_per_launch") and prof.get("l2_peak_gbs"):
        l2 = float(prof["l2_bytes_per_launch"])
        roof["l2"] = {"bytes_per_launch": l2, "achieved_gbs": l2 / t_launch / 1e9, "peak_gbs": prof["l2_peak_gbs"],
                      "frac": l2 / t_launch / 1e9 / prof["l2_peak_gbs"],
                      "source": "ncu lts__t_sectors of one launch (profiles/traffic.json); peak = the "
                                "counter's peak sector rate x 32 B"}

    # K0 (channel-data preparation): acquisition order -> frame-contiguous layout, per
    # storage type; HBM-bound, so it is reported against the measured copy bandwidth
    k0 = {}
    if True:
        T_, C_, S_, F_ = acq.iq_shape
        scanner = iq_c64.permute(3, 0, 1, 2).contiguous()
        n = scanner.numel()
        for dt, ob in (("c64", 8), ("c64split", 8), ("f16x2", 4), ("bf16x2", 4)):
            out = m.prepare_iq(scanner, "ftcs", dt)
            for _ in range(3):
                m.mach_iq_convert(scanner, "ftcs", out, dt, T_, C_, S_, F_)
            ts = []
            for _ in range(20):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                m.mach_iq_convert(scanner, "ftcs", out, dt, T_, C_, S_, F_)
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1) / 1e3)
            t = statistics.median(ts)
            byts = n * (8 + ob)
            k0[dt] = {"ms": t * 1e3, "bytes": byts, "achieved_gbs": byts / t / 1e9, "peak_gbs": hbm_peak,
                      "frac": byts / t / 1e9 / hbm_peak}
        del scanner, out

    # the same step on interleaved complex64 rows, for comparison with the split layout
    alt = {}
    if args.iq_dtype == "c64split" and not args.variant:
        acq_i = acq.replace(iq_dtype="c64")
        with m.Plan(**m.plan_kwargs(acq_i)) as pi:
            for _ in range(args.warmup):
                flush.zero_()
                m.mach_power_doppler(pi.handle, iq_c64, pd, y)
            ts = []
            for _ in range(min(args.steps, 1000)):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                m.mach_power_doppler(pi.handle, iq_c64, pd, y)
                e1.record(stream)
                ts.append((e0, e1))
            torch.cuda.synchronize()
            tt = statistics.mean(a.elapsed_time(b) for a, b in ts) / 1e3
            alt["c64_interleaved"] = {"value": acq.points / tt, "ms_per_step": tt * 1e3,
                                      "variant": pi.info()["variant"]}
        # the same step reading every term from a plan-time table (mach_das_desc.term_table)
        # instead of evaluating it (or, when that is the timed plan, the on-the-fly one), and
        # the check that both give the same bits
        try:
            pt = m.Plan(**m.plan_kwargs(acq), term_table=not args.term_table)
        except m.MachError as e:
            alt["term_table"] = {"unavailable": str(e)}
        else:
            with pt:
                pd_t = torch.empty_like(pd)
                y_t = torch.empty_like(y)
                for _ in range(args.warmup):
                    flush.zero_()
                    m.mach_power_doppler(pt.handle, iq, pd_t, y_t)
                ts = []
                for _ in range(min(args.steps, 1000)):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    m.mach_power_doppler(pt.handle, iq, pd_t, y_t)
                    e1.record(stream)
                    ts.append((e0, e1))
                torch.cuda.synchronize()
                tt = statistics.mean(a.elapsed_time(b) for a, b in ts) / 1e3
                m.mach_power_doppler(plan.handle, iq, pd, y)
                torch.cuda.synchronize()
                ti = pt.info()
                alt["on_the_fly_delays" if args.term_table else "term_table"] = {
                                     "value": acq.points / tt, "ms_per_step": tt * 1e3, "variant": ti["variant"],
                                     "table_bytes": ti["term_table_bytes"],
                                     "bitwise_equal": bool(torch.equal(y_t, y) and torch.equal(pd_t, pd))}

    # end to end through the public API with host buffers (pinned), copies timed: the host
    # holds complex64 IQ in acquisition order; each step copies one acquisition in,
    # converts it (K0), beamforms it and copies its frames and Power Doppler out.  The
    # headline uses the native pipelined entry point (upload of k+1 overlapping the compute
    # of k and the download of k-1) over a ring of distinct host buffers; the one-call-per-
    # acquisition path, which serialises copies and compute, is reported beside it
    e2e = None
    if args.e2e_steps > 0:
        ring = 4
        iq_host = iq_c64.permute(3, 0, 1, 2).contiguous().cpu()
        iq_pin = [iq_host.clone().pin_memory() for _ in range(ring)]
        pd_pin = [torch.empty(V, dtype=torch.float32).pin_memory() for _ in range(ring)]
        y_pin = [torch.empty((V, F), dtype=torch.complex64).pin_memory() for _ in range(ring)]
        K = args.e2e_steps
        seq_iq = [iq_pin[k % ring] for k in range(K)]
        seq_pd = [pd_pin[k % ring] for k in range(K)]
        seq_y = [y_pin[k % ring] for k in range(K)]
        plan.power_doppler_host_stream(seq_iq[:ring], seq_pd[:ring], seq_y[:ring], order="ftcs")
        barrier()
        t0 = time.perf_counter()
        plan.power_doppler_host_stream(seq_iq, seq_pd, seq_y, order="ftcs")
        te = shard.max_over_ranks(time.perf_counter() - t0)
        for _ in range(3):
            plan.power_doppler_host(iq_pin[0], pd_pin[0], y_pin[0], order="ftcs")
        barrier()
        t0 = time.perf_counter()
        for _ in range(K):
            plan.power_doppler_host(iq_pin[0], pd_pin[0], y_pin[0], order="ftcs")
        ts = shard.max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": world * acq.points * K / te, "unit": UNIT,
               "h2d_bytes_per_step": iq_host.numel() * iq_host.element_size(),
               "d2h_bytes_per_step": V * 4 + V * F * 8, "steps": K,
               "api": "mach_power_doppler_host_stream (pipelined, 2 staging sets, 3 streams)",
               "sequential": {"value": world * acq.points * K / ts, "unit": UNIT,
                              "api": "mach_iq_convert + mach_power_doppler per call, synchronised"}}

    # the CPU baseline leg: the oracle timed on a bounded sample, and the timed output
    # checked against it on sampled voxels (contract and exact, all-FP64, delays)
    cpu = err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(acq, iq_c64.cpu(), args.cpu_seconds)
        m.mach_power_doppler(plan.handle, iq, pd, y)
        err = oracle_error(acq, iq_c64, y, pd, 1024)

    # the other workloads, each in its own timed region on the same GPU (rank 0, one GPU):
    # the largest single-GPU configuration (the 128^3 matrix-array volume), the one-frame
    # B-mode configuration and the ragged batch
    extra = {}
    if rank == 0 and world == 1 and not args.no_extra:
        del iq_c64
        for name, dt, st in (("volume3d", "c64split", 5), ("bmode2d", "c64", 300)):
            a2, iq2 = synth.make(name, "full", device=dev)
            extra[name] = das_leg(a2, iq2, dt, st, 3, flush, stream, cpu_check=not args.no_cpu_baseline)
            del iq2
            torch.cuda.empty_cache()
        extra["ragged"] = ragged_leg(args, flush)
        torch.cuda.empty_cache()
        # learned compounding (3-angle DAS + U-Net against plain 21-angle DAS, 64 scenes at 128^3)
        la = argparse.Namespace(**{**vars(args), "steps": 3, "warmup": 3, "no_cpu_baseline": True})
        extra["learned3d"] = run_learned(la, print_line=False)
        torch.cuda.empty_cache()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if args.iq_dtype in ("c64", "c64split") else f"f32 ({args.iq_dtype} IQ storage)",
                "data": "synthetic",
                "config": workload_config(acq, {"parallelism": f"replicas{world}",
                                                "iq_layout": {"c64split": "complex64 values, each sample row split "
                                                              "into F real then F imaginary parts (K0 output)",
                                                              "c64": "interleaved complex64"}.get(args.iq_dtype,
                                                                                                  args.iq_dtype),
                                                "kernel_variant": info["variant"],
                                                "delays": ("term table (every term evaluated at plan time)"
                                                           if args.term_table else
                                                           "hybrid: transmit table + receive delays on the fly"),
                                                "active_fraction": active_terms / (V * acq.n_elem * acq.n_tx)}),
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "plan": info, "k0_iq_convert": k0,
                "error_db_vs_oracle": err, "workloads": extra,
                "other_layouts": alt,
                "gpu_launches": launches_per_step * args.steps,
                "clocks": clk, "wall_s_timed_region": t_wall,
                "paper_context": {"points_per_s": PAPER_POINTS_PER_S,
                                  "what": "Sec. 4.2: 0.23 ms on an RTX 5090 for the 251x251 px "
                                          "PyMUST rotating-disk dataset (not this exact workload)",
                                  "ratio": value / PAPER_POINTS_PER_S}}
        print(json.dumps(line))
    plan.close()


# ------------------------------------------------------------- ragged batch ----

def run_ragged(args):
    """64 seeded instances (2D and 3D, 1-48 frames, 1-15 transmits, float16 IQ) in one
    persistent launch: default shapes, autotuned shapes, and the same instances beamformed
    one plan after another."""
    import torch
    import synth
    from synth.ragged import ragged_instances
    import paper_2604_06257_gb300 as m
    from paper_2604_06257_gb300 import autotune, build as pkg_build

    pkg_build.build()
    m.lib()
    acqs = ragged_instances(n=args.ragged_n, seed=4, iq_dtype="f16x2", scale=args.ragged_scale)
    kws = [m.plan_kwargs(a) for a in acqs]
    iqs, ys, pds = [], [], []
    for i, a in enumerate(acqs):
        iqs.append(synth.iqmod.to_f16x2(synth.random_iq(a, 1000 + i, device="cuda")))
        ys.append(torch.empty((a.n_vox, a.n_frames), dtype=torch.complex64, device="cuda"))
        pds.append(torch.empty(a.n_vox, dtype=torch.float32, device="cuda"))
    points = sum(a.points for a in acqs)

    def timed(fn, steps):
        for _ in range(max(1, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3 / steps

    steps = max(1, min(args.steps, 10))
    out = {}
    with m.Batch(kws) as b:
        b.bind(iqs, ys, pds)
        t_def = timed(b.run, steps)
        out["batch_default"] = {"s": t_def, "value": points / t_def, "info": {k: v for k, v in b.info().items()
                                                                              if k != "shapes"}}
    t0 = time.perf_counter()
    shapes = None if args.no_autotune else autotune.tune_batch(kws, iqs, ys, pds)
    t_tune = time.perf_counter() - t0
    with m.Batch(kws, shapes=shapes) as b:
        b.bind(iqs, ys, pds)
        t_tuned = timed(b.run, steps)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            b.run()
        t_graph = timed(g.replay, steps)
    plans = [m.Plan(**kw) for kw in kws]

    def seq():
        for pl, iq, y, pd in zip(plans, iqs, ys, pds):
            m.mach_power_doppler(pl.handle, iq, pd, y)
    t_seq = timed(seq, steps)
    for pl in plans:
        pl.close()
    line = {"metric": "ragged batch DAS points/s (Eq. 1 summed over 64 instances)", "value": points / t_graph,
            "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": args.warmup, "ms_per_step": t_graph * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f16x2 IQ storage)",
            "data": "synthetic",
            "config": {"workload": f"{len(acqs)} seeded instances: 2D 64-256 el / 128^2-384^2 px and 3D "
                                   f"256-1024 el / 64^3-112^3 voxels (grid scale {args.ragged_scale}), 1-48 "
                                   "frames, 1-15 transmits, log-uniform sizes (seed 4)",
                       "points_per_step": points, "autotune_s": t_tune,
                       "autotuned": shapes is not None,
                       "note": "the autotuner keeps per-instance shapes only if the whole batch runs faster"},
            "batch_graph_autotuned": {"s": t_graph, "value": points / t_graph},
            "batch_autotuned": {"s": t_tuned, "value": points / t_tuned},
            **out,
            "sequential_plans": {"s": t_seq, "value": points / t_seq}}
    print(json.dumps(line))


# ------------------------------------------------------- learned compounding ----

def run_learned(args, print_line=True):
    """Learned compounding at 128^3 (matrix array, 1024 elements, 64 scenes per batch on the
    frame axis, split complex64 IQ rows for both paths): 3-angle DAS followed by the
    trained U-Net, against plain 21-angle DAS of the same scenes.  Value = volumes/s of
    the learned path; both paths' errors against the 21-angle volumes on held-out scenes
    are reported with it."""
    import numpy as np
    import torch
    import oracle
    from oracle import unet_oracle
    import paper_2604_06257_gb300 as m
    from paper_2604_06257_gb300 import build as pkg_build, learned as Lc
    from paper_2604_06257_gb300.nn import UNet
    from synth import phantoms
    from synth.iq import simulate_frames

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU fallback)")
    pkg_build.build()
    m.lib()
    n, B, nblk = 128, 64, 64
    V = n ** 3
    params, gain, levels, base, coords = Lc.load(os.path.join(Lc.WEIGHTS_DIR, "unet_few3_many21_128.npz"))
    # held-out scenes: blocks never used in training, complex-weighted, one scene per frame
    acq_blk = Lc.acquisition(n, nblk, "many")
    seeds = range(Lc.TEST_SEED0 + 5000, Lc.TEST_SEED0 + 5000 + nblk)
    iq_blk = simulate_frames(acq_blk, [phantoms.compounding_base(acq_blk, s) for s in seeds], "cuda")
    T, C, S, _ = iq_blk.shape
    Wsc = torch.as_tensor(Lc.scene_weights(np.random.default_rng(99), nblk, B)).cuda()
    iq = (iq_blk.view(-1, nblk) @ Wsc).view(T, C, S, B).contiguous()
    del iq_blk
    # the scanner's order [F][T][C][S] for the end-to-end leg; the kernels' split rows
    # (K0, outside the timed region) for the device-resident legs
    few_scanner = iq.index_select(0, torch.tensor(Lc.FEW_IN_MANY, device="cuda")).permute(3, 0, 1, 2).contiguous()
    iq_few = m.prepare_iq(few_scanner, "ftcs", "c64split")
    iq = m.prepare_iq(iq.permute(3, 0, 1, 2).contiguous(), "ftcs", "c64split")
    acq_many = Lc.acquisition(n, B, "many").replace(iq_dtype="c64split")
    acq_few = Lc.acquisition(n, B, "few").replace(iq_dtype="c64split")
    pm, pf = m.Plan(**m.plan_kwargs(acq_many)), m.Plan(**m.plan_kwargs(acq_few))
    net = UNet(n, n, n, B, levels=levels, base_ch=base, inference_only=True, coords=coords)
    net.set_params(params)
    net.set_gain(gain)
    y_many = torch.empty((V, B), dtype=torch.complex64, device="cuda")
    y_few = torch.empty_like(y_many)
    pred = torch.empty_like(y_many)
    flush = L2Flush("cuda")
    stream = torch.cuda.current_stream()

    def plain():
        pm.run(iq, y_many)

    def learned():
        pf.run(iq_few, y_few)
        net.forward(y_few, pred)

    def unet_only():
        net.forward(y_few, pred)

    plain()
    learned()
    torch.cuda.synchronize()
    err = {"network_vs_21_angle_db": Lc.nrmse_db(pred, y_many),
           "few_angle_ls_gain_vs_21_angle_db": Lc.nrmse_db(gain * y_few, y_many),
           "target_db": -30.0, "scenes": B, "blocks": nblk,
           "scenes_recipe": "complex-weighted sums of 6-16 seeded blocks (speckle patch / point cluster / "
                            "vessel) never used in training"}

    def timed(fn, steps):
        for _ in range(max(3, args.warmup)):
            flush.zero_()
            fn()
        evs = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return statistics.mean(a.elapsed_time(b) for a, b in evs) / 1e3

    steps = max(1, min(args.steps, 20))
    clocks = Clocks(torch.cuda.get_device_properties(0).uuid.__str__())
    clocks.start()
    t_learned = timed(learned, steps)
    t_plain = timed(plain, steps)
    t_unet = timed(unet_only, steps)
    clk = clocks.stop()
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("bf16_tflops", 1900.0)
    achieved = net.flops_forward * B / t_unet / 1e12
    L = levels
    unet_launches = 2 + (L - 1) + 2 * L + 4 * (L - 1) + 2

    # end to end through the public API: the 3-angle IQ in the scanner's order from pinned
    # host memory, K0 to split rows, DAS, U-Net, the prediction back to pinned host
    # memory; copies inside the timed region.  Two staging sets and separate upload /
    # download streams let step k+1's upload and step k-1's download overlap step k's
    # beamforming and network (events order the reuse of each set)
    iq_pin = few_scanner.cpu().pin_memory()
    out_pin = torch.empty((V, B), dtype=torch.complex64).pin_memory()
    scan_dev = [torch.empty_like(few_scanner) for _ in range(2)]
    pred2 = [pred, torch.empty_like(pred)]
    Tf = len(Lc.FEW_IN_MANY)
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    ev = {k: [torch.cuda.Event(), torch.cuda.Event()] for k in ("up", "read", "done", "down")}
    state = {"k": 0}

    def e2e_step():
        b = state["k"] % 2
        state["k"] += 1
        with torch.cuda.stream(up):
            up.wait_event(ev["read"][b])            # K0 of step k-2 has read this set
            scan_dev[b].copy_(iq_pin, non_blocking=True)
            ev["up"][b].record(up)
        stream.wait_event(ev["up"][b])
        m.mach_iq_convert(scan_dev[b], "ftcs", iq_few, "c64split", Tf, C, S, B, stream)
        ev["read"][b].record(stream)
        pf.run(iq_few, y_few, stream)
        stream.wait_event(ev["down"][b])            # step k-2's prediction has been read back
        net.forward(y_few, pred2[b], stream)
        ev["done"][b].record(stream)
        with torch.cuda.stream(down):
            down.wait_event(ev["done"][b])
            out_pin.copy_(pred2[b], non_blocking=True)
            ev["down"][b].record(down)

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        e2e_step()
    torch.cuda.synchronize()
    t_e2e = (time.perf_counter() - t0) / steps

    # the oracle (FP64 C DAS + numpy U-Net) on one 64^3 sub-volume of one scene, scaled to
    # whole volumes by the voxel count (both stages cost in proportion to the voxels)
    cpu = None
    if not args.no_cpu_baseline:
        h = n // 2
        sub = acq_few.replace(n_frames=1, iq_dtype="c64")
        iq1 = few_scanner[:1].permute(1, 2, 3, 0).contiguous().cpu()
        g = np.arange(h) + h // 2
        idx = (g[None, None, :] + n * (g[None, :, None] + n * g[:, None, None])).ravel()
        t0 = time.perf_counter()
        y1, _ = oracle.das(sub, iq1, idx)
        t_das = time.perf_counter() - t0
        t0 = time.perf_counter()
        unet_oracle.forward(params.astype(np.float64), y1, (h, h, h), levels, base, gain)
        t_net = time.perf_counter() - t0
        per_vol = (t_das + t_net) * (V / len(idx))
        cpu = {"value": 1.0 / per_vol, "unit": "volumes/s", "cores": oracle.max_threads(), "kind": "oracle",
               "sample": f"one 64^3 sub-volume of one scene: FP64 3-angle DAS {t_das:.1f} s + FP64 U-Net "
                         f"{t_net:.1f} s, scaled by the voxel count ({V // len(idx)}x) to a 128^3 volume"}
    line = {"metric": "compounded 128^3 volumes/s: 3-angle DAS + learned U-Net (vs plain 21-angle DAS)",
            "value": B / t_learned, "unit": "volumes/s", "n_gpus": 1, "steps": steps, "warmup": max(3, args.warmup),
            "ms_per_step": t_learned * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 DAS, bf16 U-Net (f32 accumulate)", "data": "synthetic",
            "config": {"workload": f"learned compounding: 32x32 matrix array (1024 el, fc 7.8 MHz, fs 31.2 MHz), "
                                   f"{n}^3 voxels at 0.1 mm, {B} scenes per batch (frame axis, split complex64 IQ "
                                   "rows for both paths), 3 plane waves "
                                   "(az -10/0/10 deg) + U-Net (4 levels, 16-128 ch, 3x3x3, bf16) vs 21 plane "
                                   "waves (az/el cross, -10..10 deg)",
                       "l2": "flushed between timed steps (256 MB write, then 256 MB read, outside the timed events)",
                       "weights": "unet_few3_many21_128.npz (trained by paper_2604_06257_gb300.learned)"},
            "plain_21_angle": {"value": B / t_plain, "ms_per_step": t_plain * 1e3, "variant": pm.info()["variant"],
                               "points_per_s": acq_many.points / t_plain},
            "speedup_vs_plain": t_plain / t_learned,
            "few_angle_das_ms": (t_learned - t_unet) * 1e3, "unet_forward_ms": t_unet * 1e3,
            "error_db": err,
            "roofline": {"bound": "tensor", "kernel": "U-Net forward (k_conv3d implicit GEMMs + elementwise)",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": None, "peak_source": "bf16 dense, MEASURED_PEAKS.json (burst)",
                         "algorithmic": f"{net.flops_forward / 1e9:.1f} GFLOP per volume (2 x 27 x Cin x Cout "
                                        "per voxel per convolution)"},
            "cpu_baseline": cpu,
            "e2e": {"value": B / t_e2e, "unit": "volumes/s",
                    "h2d_bytes_per_step": iq_pin.numel() * iq_pin.element_size(),
                    "d2h_bytes_per_step": out_pin.numel() * out_pin.element_size(), "steps": steps},
            "gpu_launches": (1 + unet_launches) * steps, "clocks": clk}
    net.close()
    pm.close()
    pf.close()
    if print_line:
        print(json.dumps(line))
    return line


# ------------------------------------------------------------ scaling sweep ----

def run_sweep(args):
    """Throughput against voxels, channels and frames (the scaling study of Sec. 4.6,
    Fig. 5), one JSON line per point, on the 2D Doppler geometry (one 0-degree plane wave,
    fc 5.2 MHz, fs 20.8 MHz, 2048 samples, F# 1.0) with seeded random IQ (the values do not
    change the work):
      voxels   63 k - 6.3 M: the same 25.6 x 25.6 mm field of view sampled by n x n pixels;
      channels 128 - 8192: the same 38.4 mm linear aperture with C elements (pitch 38.4 mm / C),
               so each voxel keeps the same share of active elements;
      frames   1 - 512: the 256 x 256 grid, 128 elements.
    Split complex64 rows where F is a multiple of 4 above 4, interleaved complex64 otherwise;
    the plan's default kernel for each point."""
    import numpy as np
    import torch
    import synth
    import paper_2604_06257_gb300 as m
    from paper_2604_06257_gb300 import build as pkg_build
    from synth.acquisition import linear_array

    pkg_build.build()
    m.lib()
    flush = L2Flush("cuda")
    stream = torch.cuda.current_stream()
    base = synth.doppler2d()
    fov = 25.6e-3

    def point(axis, value, acq):
        F = acq.n_frames
        dt = "c64split" if F % 4 == 0 and F > 4 else "c64"
        iq = synth.random_iq(acq, 7, device="cuda")
        est = 2e-12 * acq.points + 2e-5                       # rough seconds per step
        steps = int(min(500, max(3, 0.5 / est)))
        leg = das_leg(acq, iq, dt, steps, 3, flush, stream, cpu_check=False)
        del iq
        torch.cuda.empty_cache()
        line = {"metric": METRIC, "sweep": axis, axis: value, "value": leg["value"], "unit": UNIT,
                "ms_per_step": leg["ms_per_step"], "steps": steps, "variant": leg["variant"], "dtype": dt,
                "higher_is_better": True, "data": "synthetic", "config": leg["config"],
                "roofline": leg["roofline"]}
        print(json.dumps(line), flush=True)

    axes = args.sweep_axes.split(",")
    if "voxels" in axes:
        for n in (251, 512, 1024, 1448, 2048, 2510):
            step = fov / n
            acq = base.replace(grid_dims=(n, 1, n), grid_origin=(-(n - 1) * step / 2, 0.0, 10e-3),
                               grid_step=(step, 0.0, step), name=f"sweep_vox{n * n}")
            point("voxels", n * n, acq)
    if "channels" in axes:
        for C in (128, 256, 512, 1024, 2048, 4096, 8192):
            acq = base.replace(elem_pos=linear_array(C, pitch=38.4e-3 / C), name=f"sweep_ch{C}")
            point("channels", C, acq)
    if "frames" in axes:
        for F in (1, 2, 4, 8, 16, 32, 64, 128, 256, 512):
            acq = base.replace(n_frames=F, name=f"sweep_f{F}")
            point("frames", F, acq)


# ---------------------------------------------------------- reference arm ----

def run_reference(args):
    import numpy as np
    import torch
    import synth
    import oracle

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    if torch.cuda.is_available():
        acq, iq = synth.make(args.workload, "full", device="cuda")
        iq_host = iq.cpu()
        del iq
        src = "seeded synthetic IQ (generated on the GPU, copied to host)"
    else:
        acq = synth.make_acquisition(args.workload, "full")
        iq_host = synth.random_iq(acq, 0)
        src = "seeded complex Gaussian IQ (no GPU to synthesise the phantom)"
    budget = 120.0                                     # whole run within about two minutes
    per_step = min(20.0, max(0.02, budget / max(1, args.steps + args.warmup)))
    cal = np.arange(0, acq.n_vox, max(1, acq.n_vox // 256))[:256]
    t = time.perf_counter()
    oracle.das(acq, iq_host, cal, want_y=False)
    dt = max(time.perf_counter() - t, 1e-6)
    n = int(min(acq.n_vox, max(16, len(cal) * per_step / dt)))
    idx = np.linspace(0, acq.n_vox - 1, n).astype(np.int64)
    for _ in range(args.warmup):
        oracle.das(acq, iq_host, idx, want_y=True)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.das(acq, iq_host, idx, want_y=True)
        times.append(time.perf_counter() - t)
    pts = n * acq.n_elem * acq.n_tx * acq.n_frames
    value = pts / statistics.mean(times)
    cores = oracle.max_threads()
    sample = (f"{n} of {acq.n_vox} voxels (evenly strided) per step, all channels, transmits and "
              f"frames, FP64, {src}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(times) * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(acq, {"parallelism": "host cores (OpenMP)"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_rf(args):
    """RF input on the 2D Power Doppler geometry: real RF at 4x the IQ rate (83.2 MHz, 8189
    samples per channel and frame) demodulated, low-passed (32 taps) and decimated into the
    complex64 IQ the beamformer reads (mach_rf_to_iq), then beamformed with Power Doppler.
    Timed: the demodulation alone, and demodulation + beamforming per acquisition."""
    import torch
    import synth
    import paper_2604_06257_gb300 as m
    from paper_2604_06257_gb300 import build as pkg_build
    from synth.iq import lowpass_taps

    pkg_build.build()
    m.lib()
    acq = synth.make_acquisition("doppler2d", "full", "c64")
    decim, L = 4, 32
    T, C, S, F = acq.iq_shape
    S_rf = decim * (S - 1) + 1
    fs_rf = acq.fs * decim
    g = torch.Generator(device="cuda")
    g.manual_seed(7)
    rf = torch.randn((T, C, S_rf, F), generator=g, device="cuda")   # values do not change the timing
    taps = lowpass_taps(L, acq.fc, fs_rf)
    iq = torch.empty((T, C, S, F), dtype=torch.complex64, device="cuda")
    plan = m.Plan(**m.plan_kwargs(acq))
    pd = torch.empty(acq.n_vox, dtype=torch.float32, device="cuda")
    y = torch.empty((acq.n_vox, F), dtype=torch.complex64, device="cuda")
    flush = L2Flush("cuda")
    stream = torch.cuda.current_stream()

    def demod():
        m.mach_rf_to_iq(rf, taps, fs_rf, acq.fc, acq.t0, decim, iq)

    def both():
        demod()
        m.mach_power_doppler(plan.handle, iq, pd, y)

    def timed(fn, steps):
        for _ in range(max(3, args.warmup)):
            flush.zero_()
            fn()
        evs = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return statistics.mean(a.elapsed_time(b) for a, b in evs) / 1e3

    steps = max(1, min(args.steps, 500))
    t_demod = timed(demod, steps)
    t_both = timed(both, steps)
    n_iq = T * C * S * F
    byts = 4 * T * C * S_rf * F + 8 * n_iq                 # RF read once, IQ written once
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    line = {"metric": "DAS points/s from RF input (demodulation + beamforming + Power Doppler)",
            "value": acq.points / t_both, "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": args.warmup,
            "ms_per_step": t_both * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{acq.name} from RF: {S_rf} RF samples per channel and frame at "
                                   f"{fs_rf / 1e6:.1f} MHz, {L}-tap low-pass, decimation {decim}",
                       "l2": "flushed between steps (256 MB write, then 256 MB read)"},
            "demodulation": {"ms": t_demod * 1e3, "iq_samples_per_s": n_iq / t_demod,
                             "bytes": byts, "achieved_gbs": byts / t_demod / 1e9, "peak_gbs": hbm,
                             "frac": byts / t_demod / 1e9 / hbm},
            "gpu_launches": 2 * steps}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "ragged":
        run_ragged(args)
    elif args.workload == "learned3d":
        run_learned(args)
    elif args.workload == "rf2d":
        run_rf(args)
    elif args.workload == "sweep":
        run_sweep(args)
    else:
        run_ours(args)
    try:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()
    except Exception:
        pass


if __name__ == "__main__":
    main()
