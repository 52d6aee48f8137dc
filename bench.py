#!/usr/bin/env python3
"""Throughput bench of libfalcon on the 67,108,864-value segment workload.

One step = compress + decompress of the FP64 array and of the FP32 array (four kernel
launches), inputs resident in HBM.  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl falcon|reference]

Under torchrun each rank runs its own replica on its own GPU (chunks are independent:
weak scaling, no collective on the data path); value = bytes of all ranks / max time.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_VALUES = 1 << 26
BLOCK = 1024
METRIC = "comp/decomp GB/s & % HBM peak, bit-exact; batched vs plain; serve p99 ms"
WORKLOAD = ("segments: 67,108,864 values, once FP64 and once FP32; 4096-value segments with "
            "0..6 decimal places, sinusoid amplitude 10^U(0,4) + AR(1) noise, 1% full-precision "
            "outliers, 0.01% NaN/inf/subnormal/-0; block 1024")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="falcon", choices=["falcon", "reference"])
    ap.add_argument("--n", type=int, default=N_VALUES, help=argparse.SUPPRESS)
    ap.add_argument("--section", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--kernels-only", action="store_true",
                    help="only the timed kernel steps (every other section off; used by the ncu captures)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-pipeline", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-case1", action="store_true")
    ap.add_argument("--no-f16", action="store_true")
    ap.add_argument("--no-analytics", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-schedulers", action="store_true")
    ap.add_argument("--no-sweeps", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help=argparse.SUPPRESS)
    ap.add_argument("--serve-seconds-saturated", type=float, default=3.0, help=argparse.SUPPRESS)
    ap.add_argument("--serve-pool", type=int, default=256, help=argparse.SUPPRESS)
    ap.add_argument("--serve-rates", default="1000,2000,5000,10000,20000,50000", help=argparse.SUPPRESS)
    ap.add_argument("--pipeline-values", type=int, default=1 << 31, help=argparse.SUPPRESS)
    ap.add_argument("--batch-series", type=int, default=4096, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.kernels_only:
        for k in ("no_cpu_baseline", "no_e2e", "no_batched", "no_pipeline", "no_serve", "no_case1", "no_f16",
                  "no_analytics", "no_variants", "no_schedulers", "no_sweeps"):
            setattr(args, k, True)
    return args


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class NvmlSampler:
    """Samples the SM clock and the clock-event (throttle) reasons through NVML (the driver's
    libnvidia-ml, loaded with ctypes) every few milliseconds while the timed region runs, so
    that even a short region is covered.  Read-only queries."""

    # nvmlClocksEventReasons bits
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    NVML_CLOCK_SM = 1

    def __init__(self, index: int, pci_bus: str | None = None, period_s: float = 0.002):
        import ctypes
        self.ct = ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.lib = lib
        self.handle = ctypes.c_void_p()
        # the CUDA device's own GPU (by PCI address), else NVML's device `index`
        found = pci_bus is not None and lib.nvmlDeviceGetHandleByPciBusId_v2(
            pci_bus.encode(), ctypes.byref(self.handle)) == 0
        if not found and lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.handle)) != 0:
            raise RuntimeError("no NVML handle")
        self.reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint()
        self.max_mhz = float(mx.value) if lib.nvmlDeviceGetMaxClockInfo(
            self.handle, self.NVML_CLOCK_SM, ctypes.byref(mx)) == 0 else None
        self.period = period_s
        self.samples = []
        self.recording = False
        self.stop_flag = False
        self.thread = None

    def _one(self):
        ct = self.ct
        mhz, rs = ct.c_uint(), ct.c_ulonglong()
        if self.lib.nvmlDeviceGetClockInfo(self.handle, self.NVML_CLOCK_SM, ct.byref(mhz)) != 0:
            return None
        if self.reasons_fn(self.handle, ct.byref(rs)) != 0:
            return None
        return float(mhz.value), int(rs.value)

    def _run(self):
        while not self.stop_flag:
            if self.recording:
                s = self._one()
                if s is not None:
                    self.samples.append(s)
            time.sleep(self.period)

    def start(self):
        if self.thread is None:
            self.thread = threading.Thread(target=self._run, daemon=True)
            self.thread.start()

    def __enter__(self):
        self.start()
        self.samples.clear()
        first = self._one()                      # one sample at the start of the region
        if first is not None:
            self.samples.append(first)
        self.recording = True
        return self

    def __exit__(self, *exc):
        self.recording = False
        last = self._one()                       # and one at its end
        if last is not None:
            self.samples.append(last)
        self.stop_flag = True
        if self.thread is not None:
            self.thread.join(timeout=2)

    def summary(self):
        sm = [m for m, _ in self.samples]
        reasons = set()
        for _, r in self.samples:
            for bit, nm in self.REASONS.items():
                if r & bit:
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.max_mhz,
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvml"}


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs
    (used where NVML cannot be loaded)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        self.start()
        self.lines.clear()
        return self

    def start(self):
        if self.proc is not None:
            return
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t0 = time.time()                     # let nvidia-smi come up before timing
            while not self.lines and time.time() - t0 < 5:
                time.sleep(0.05)
            self.lines.clear()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi"}


def clock_sampler(index: int):
    """NVML sampler if the driver's library loads, else the nvidia-smi one."""
    try:
        import torch
        pr = torch.cuda.get_device_properties(index)
        bus = f"{pr.pci_domain_id:08X}:{pr.pci_bus_id:02X}:{pr.pci_device_id:02X}.0"
    except Exception:
        bus = None
    try:
        return NvmlSampler(index, bus)
    except Exception:
        return ClockSampler(index)


# ------------------------------------------------------------------------------ reference arm
def run_reference(args):
    """The CPU oracle (the method's plain definition) timed on the host cores (its threaded
    driver over chunk ranges), on the same workload; rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle
    from paper_2511_04140_gb300 import synth
    oracle.build()
    a64 = synth.segments(args.n, seed=1)
    a32 = synth.segments(args.n, seed=1, dtype=np.float32)
    orig = a64.nbytes + a32.nbytes
    cores = host_cores()
    steps = max(1, min(args.steps, 5))               # each step is seconds of CPU work

    def step():
        for a in (a64, a32):
            s = oracle.compress(a, BLOCK, threads=cores)
            oracle.decompress(s, threads=cores)

    for _ in range(min(args.warmup, 1)):
        step()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    dt = (time.perf_counter() - t0) / steps
    gbs = 2 * orig / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": steps, "warmup": min(args.warmup, 1), "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64/int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": args.n, "block": BLOCK},
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle",
                             "sample": f"the whole workload ({args.n} FP64 + {args.n} FP32 values), compress + "
                                       f"decompress, {cores} threads over chunk ranges, {steps} steps"},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def host_cores() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(host):
    """The oracle on the host cores: one thread on the first 2^20 values of each array, and
    every core (the oracle's threaded driver over chunk ranges) on the whole arrays."""
    from oracle import oracle
    oracle.build()
    arrays = (host[np.float64], host[np.float32])
    n = len(arrays[0])

    def run(arrs, threads):
        t0 = time.perf_counter()
        for a in arrs:
            st = oracle.compress(a, BLOCK, threads=threads)
            oracle.decompress(st, threads=threads)
        return time.perf_counter() - t0

    sample = 1 << 20
    part = [a[:sample].copy() for a in arrays]
    dt1 = run(part, 1)
    cores = host_cores()
    dtn = run(arrays, cores)
    orig_part = sum(a.nbytes for a in part)
    orig = sum(a.nbytes for a in arrays)
    return {"value": 2 * orig / dtn / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"the whole workload ({n} FP64 + {n} FP32 values), compress + decompress, "
                      f"{cores} threads over chunk ranges, {dtn:.1f} s",
            "single_thread": {"value": 2 * orig_part / dt1 / 1e9, "unit": "GB/s", "cores": 1,
                              "sample": f"first {sample} values of the FP64 and of the FP32 array, "
                                        f"compress + decompress, {dt1:.1f} s"}}


def release_caches(torch):
    """Return cached device and pinned host blocks between bench sections (torch's pinned-host
    cache rounds blocks up to powers of two and otherwise keeps them for the process)."""
    import gc
    gc.collect()
    torch.cuda.empty_cache()
    getattr(torch._C, "_host_emptyCache", lambda: None)()


def profiled_traffic(kernel: str):
    """DRAM bytes per call of `kernel` from the committed ncu summary, or None when the
    compression sources changed since the capture (the figure would no longer describe them)."""
    import re
    here = os.path.dirname(os.path.abspath(__file__))
    try:
        text = open(os.path.join(here, "profiles", "dram_traffic_segments_2e26.md")).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_call " + re.escape(kernel) + r" (\d+) sources ([0-9a-f]+)", text)
    if not m:
        return None
    return int(m.group(1)) if compress_sources_digest() == m.group(2) else None


def compress_sources_digest(root: str | None = None) -> str:
    """First 16 hex digits of sha256 over the compression kernels' sources (under `root`,
    default this repository) with comments and whitespace removed: a comment edit does not
    change the profiled kernels."""
    import hashlib
    import re
    here = root or os.path.dirname(os.path.abspath(__file__))
    h = hashlib.sha256()
    for f in ("compress.cu", "falcon_device.cuh", "falcon_internal.h", "falcon_tables.h"):
        with open(os.path.join(here, "paper_2511_04140_gb300", "csrc", f)) as fh:
            code = fh.read()
        code = re.sub(r"/\*.*?\*/", " ", code, flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        h.update(" ".join(code.split()).encode())
    return h.hexdigest()[:16]


def max_over_ranks(x: float, dist, device) -> float:
    """The largest of every rank's x (the job ends when its slowest replica does)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(step_bytes_per_rank: int, world: int, ms_per_step: float) -> float:
    """GB/s of original bytes over all replicas: each rank moves step_bytes_per_rank per step."""
    return step_bytes_per_rank * world / (ms_per_step / 1e3) / 1e9


def progress(stage):
    """One line per bench stage on stderr (elapsed seconds, peak host RSS)."""
    import resource
    rss = resource.getrusage(resource.RUSAGE_SELF).ru_maxrss / 2**20
    sys.stderr.write(f"[bench {time.perf_counter() - _T0:7.1f} s, peak rss {rss:5.1f} GiB] {stage}\n")
    sys.stderr.flush()


_T0 = time.perf_counter()


# ------------------------------------------------------------------------------ falcon arm
def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.section:
        return section_main(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    from paper_2511_04140_gb300 import build as fbuild
    fbuild.build()
    from paper_2511_04140_gb300 import falcon, synth

    n = args.n
    progress("generating inputs")
    host = {np.float64: synth.segments(n, seed=1), np.float32: synth.segments(n, seed=1, dtype=np.float32)}
    stream = torch.cuda.Stream(device=dev)
    st_ptr = stream
    bufs = {}
    for dt, arr in host.items():
        code = falcon.F64 if dt == np.float64 else falcon.F32
        x = torch.from_numpy(arr).to(dev)
        nc = (n + BLOCK - 1) // BLOCK
        cap = falcon.bound(n, code, BLOCK)
        bufs[dt] = dict(x=x, code=code, out=torch.empty(cap, dtype=torch.uint8, device=dev),
                        y=torch.empty_like(x),
                        ws_c=torch.zeros(falcon.workspace_bytes(nc), dtype=torch.uint8, device=dev),
                        ws_d=torch.zeros(falcon.workspace_bytes(nc), dtype=torch.uint8, device=dev),
                        res_c=torch.zeros(2, dtype=torch.int64, device=dev),
                        res_d=torch.zeros(2, dtype=torch.int64, device=dev))
    # stream lengths (needed by the async decompress) from one untimed call
    for dt, b in bufs.items():
        s = falcon.compress(b["x"], BLOCK, out=b["out"])
        b["nbytes"] = s.numel()
        b["header"] = s[:32].cpu().numpy().tobytes()
    torch.cuda.synchronize(dev)

    kernels = [("compress_f64", np.float64, "c"), ("decompress_f64", np.float64, "d"),
               ("compress_f32", np.float32, "c"), ("decompress_f32", np.float32, "d")]

    def step(events=None):
        for i, (name, dt, kind) in enumerate(kernels):
            b = bufs[dt]
            if events is not None:
                events[i][0].record(stream)
            if kind == "c":
                falcon.compress_async(b["x"], BLOCK, b["out"], b["ws_c"], b["res_c"], st_ptr)
            else:
                falcon.decompress_async(b["out"], b["nbytes"], b["header"], b["y"], b["ws_d"], b["res_d"], st_ptr)
            if events is not None:
                events[i][1].record(stream)

    progress("inputs resident; kernel steps")
    clocks = clock_sampler(local)
    clocks.start()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()

    ev = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in kernels]
          for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with clocks:
        torch.cuda.synchronize(dev)
        with torch.cuda.stream(stream):
            start.record(stream)
            for k in range(args.steps):
                step(ev[k])
            stop.record(stream)
        torch.cuda.synchronize(dev)
    elapsed_ms = start.elapsed_time(stop)
    if dist:
        elapsed_ms = max_over_ranks(elapsed_ms, dist, dev)

    # results and bit-exactness (outside the timed region)
    ok = True
    for dt, b in bufs.items():
        nb, stc = (int(v) for v in b["res_c"].cpu())
        nv, std = (int(v) for v in b["res_d"].cpu())
        u = torch.int64 if dt == np.float64 else torch.int32
        ok &= (stc == 0 and std == 0 and nb == b["nbytes"] and nv == n and
               torch.equal(b["y"].view(u), b["x"].view(u)))

    per = {name: [ev[k][i][0].elapsed_time(ev[k][i][1]) for k in range(args.steps)]
           for i, (name, _, _) in enumerate(kernels)}
    peak, peak_kind = measured_peaks()
    orig = {np.float64: n * 8, np.float32: n * 4}
    kstats = {}
    for name, dt, kind in kernels:
        ms = statistics.mean(per[name])
        alg = orig[dt] + bufs[dt]["nbytes"]                      # read + write, either direction
        kstats[name] = {"ms": ms, "gbs_original": orig[dt] / ms / 1e6,
                        "hbm_gbs": alg / ms / 1e6, "hbm_frac": alg / ms / 1e6 / peak,
                        "ratio": bufs[dt]["nbytes"] / orig[dt]}
    dom = max(kstats, key=lambda k: kstats[k]["ms"])
    ms_per_step = elapsed_ms / args.steps
    step_bytes = 2 * (orig[np.float64] + orig[np.float32])
    value = whole_job_rate(step_bytes, world, ms_per_step)

    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64/int32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "block": BLOCK, "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2 (512 MiB FP64 + 256 MiB FP32)"},
        "bit_exact": bool(ok),
        "gpu_launches": 8 * args.steps,                # per dtype: compress 2 kernels, decompress 2
        "kernels": kstats,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": kstats[dom]["hbm_gbs"], "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": kstats[dom]["hbm_frac"],
                     "traffic": profiled_traffic(dom) if n == (1 << 26) else None},
        "clocks": clocks.summary(),
    }
    if rank == 0 and not args.no_e2e:
        progress("end-to-end pipeline")
        line["e2e"] = e2e(falcon, torch, bufs, host, dev, args)
    if rank == 0:
        del bufs
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_case1:
        progress("case-1 workload")
        line["case1"] = bench_case1(falcon, torch, dev, n, peak)
    if rank == 0 and not args.no_f16:
        progress("fp16 workload")
        line["f16"] = bench_f16(falcon, torch, dev, n, peak)
    if rank == 0 and not args.no_analytics:
        progress("analytics on compressed data")
        line["analytics"] = bench_analytics(falcon, torch, dev, host, peak)
    if rank == 0 and not args.no_variants:
        progress("codec variants")
        line["variants"] = bench_variants(falcon, torch, dev, host)
    if rank == 0 and not args.no_batched:
        progress("batched launch")
        line["batched"] = bench_batched(falcon, synth, torch, dev, args.batch_series)
    # the host-link sections run each in a fresh process: in one long process, the state the
    # earlier sections leave behind made host <-> device copies of later ones erratic
    # (measured: the 16 GiB pipeline at 167-177 GB/s alone, 52-69 GB/s after the batched
    # section), and a user runs each such workload on its own
    for name, skip in (("pipeline", args.no_pipeline), ("schedulers", args.no_schedulers),
                       ("sweeps", args.no_sweeps), ("serve", args.no_serve)):
        if rank == 0 and not skip:
            progress(name + " (own process)")
            line[name] = run_section(name, args)
    if rank == 0 and not args.no_cpu_baseline:
        progress("cpu baseline")
        line["cpu_baseline"] = cpu_baseline(host)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    failed = failed_checks(line)
    if failed:
        sys.stderr.write("bench: bit-exactness check failed in " + ", ".join(failed) + "\n")
        sys.exit(1)


def run_section(name: str, args) -> dict:
    """Runs one bench section in a fresh Python process on this process's GPU and returns
    its result (the last JSON line it prints)."""
    cmd = [sys.executable, os.path.abspath(__file__), "--section", name,
           "--serve-seconds", str(args.serve_seconds), "--serve-seconds-saturated", str(args.serve_seconds_saturated),
           "--serve-pool", str(args.serve_pool), "--serve-rates", args.serve_rates,
           "--pipeline-values", str(args.pipeline_values)]
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    import torch
    vis, idx = os.environ.get("CUDA_VISIBLE_DEVICES"), torch.cuda.current_device()
    env["CUDA_VISIBLE_DEVICES"] = vis.split(",")[idx] if vis else str(idx)      # the same GPU, as cuda:0
    res = subprocess.run(cmd, stdout=subprocess.PIPE, text=True, env=env)
    if res.returncode != 0:
        raise RuntimeError(f"bench section {name} failed (rc {res.returncode})")
    return json.loads(res.stdout.strip().splitlines()[-1])


def section_main(args):
    """One section, alone in this process (see run_section)."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    from paper_2511_04140_gb300 import build as fbuild
    fbuild.build()
    from paper_2511_04140_gb300 import falcon, synth
    peak, _ = measured_peaks()
    if args.section == "pipeline":
        out = bench_pipeline(falcon, synth, torch, dev, args.pipeline_values)
    elif args.section == "schedulers":
        out = bench_schedulers(falcon, torch, dev)
    elif args.section == "sweeps":
        out = bench_sweeps(falcon, torch, dev, peak)
    elif args.section == "serve":
        out = bench_serve(args, dev)
    else:
        raise SystemExit(f"unknown section {args.section}")
    print(json.dumps(out), flush=True)


def failed_checks(obj, path="line"):
    """Paths of every false `bit_exact` / `oracle_equal` / `equal_to_decompress_and_reduce` key
    in the bench line: a lossless codec that lost a bit, a stream that differs from the
    oracle's, or an aggregate that differs from the decompressed values' fails the run."""
    bad = []
    if isinstance(obj, dict):
        for k, v in obj.items():
            if k in ("bit_exact", "oracle_equal", "equal_to_decompress_and_reduce") and v is False:
                bad.append(f"{path}.{k}")
            else:
                bad += failed_checks(v, f"{path}.{k}")
    elif isinstance(obj, list):
        for i, v in enumerate(obj):
            bad += failed_checks(v, f"{path}[{i}]")
    return bad


def bench_batched(falcon, synth, torch, dev, count):
    """Independent series (lengths log-uniform in [1024, 4194304], FP64 with p = 0.7 else FP32,
    per-series places and outlier rate): the batched launches of each direction, captured in a
    CUDA graph and replayed, versus one asynchronous call per series, same buffers, inputs
    resident."""
    from paper_2511_04140_gb300 import tune
    xs = synth.series_batch_cuda(count, seed=2, device=dev)
    orig = sum(x.numel() * x.element_size() for x in xs)
    nvals = sum(x.numel() for x in xs)
    sample = xs[::max(1, count // 128)]
    tuned = tune.autotune(sample, blocks=(512, 1024, 1025), compress_ctas=(0, 3), decompress_ctas=(0, 2), reps=2)
    block = tune.apply(tuned["choice"])
    comp = falcon.Batch(falcon.COMPRESS, xs, block=block)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    comp.launch(stream)
    torch.cuda.synchronize(dev)
    res = comp.results()
    streams = comp.streams()
    comp_bytes = sum(nb for nb, _ in res)
    dec = falcon.Batch(falcon.DECOMPRESS, [(s, s.numel(), s[:32].cpu().numpy().tobytes()) for s in streams])
    # each direction captured once into a CUDA graph and timed as graph replays
    graphs = []
    for b in (comp, dec):
        side = torch.cuda.Stream(dev)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            b.launch(side)
        graphs.append(g)
    tc_b = timed(graphs[0].replay)
    td_b = timed(graphs[1].replay)
    ok = all(st == 0 for _, st in res) and all(st == 0 for _, st in dec.results())
    for x, y in zip(xs, dec.outputs):
        iv = torch.int64 if x.dtype == torch.float64 else torch.int32
        ok &= torch.equal(x.view(iv), y[:x.numel()].view(iv))
    # one launch per series (asynchronous API, same outputs), per-series completion events
    ws = [torch.zeros(falcon.workspace_bytes((x.numel() + block - 1) // block), dtype=torch.uint8, device=dev) for x in xs]
    rs = torch.zeros(2 * count, dtype=torch.int64, device=dev)
    hdrs = [s[:32].cpu().numpy().tobytes() for s in streams]
    evs = [torch.cuda.Event(enable_timing=True) for _ in xs]

    def plain_c(record=False):
        for i, x in enumerate(xs):
            falcon.compress_async(x, block, comp.outputs[i], ws[i], rs[2 * i:2 * i + 2], stream)
            if record:
                evs[i].record(stream)

    def plain_d(record=False):
        for i, x in enumerate(xs):
            falcon.decompress_async(comp.outputs[i], streams[i].numel(), hdrs[i], dec.outputs[i], ws[i],
                                    rs[2 * i:2 * i + 2], stream)
            if record:
                evs[i].record(stream)

    tc_p = timed(plain_c)
    td_p = timed(plain_d)
    e0 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    plain_c(record=True)
    torch.cuda.synchronize(dev)
    lat = sorted(e0.elapsed_time(e) for e in evs)
    p = lambda q: lat[min(len(lat) - 1, int(q * len(lat)))]
    out = {"workload": f"{count} series, {nvals} values, {orig / 1e9:.2f} GB "
                       "(log-uniform lengths 1024..4194304, FP64 p=0.7 else FP32)",
           "block": block, "tuned": tuned["choice"], "ratio": comp_bytes / orig, "bit_exact": bool(ok),
           "batched": {"compress_ms": tc_b, "decompress_ms": td_b, "gbs": 2 * orig / ((tc_b + td_b) * 1e6),
                       "form": "one CUDA graph per direction (compress: 2 kernels, decompress: 2, over all series)",
                       "p50_ms": tc_b, "p99_ms": tc_b},
           "plain": {"compress_ms": tc_p, "decompress_ms": td_p, "gbs": 2 * orig / ((tc_p + td_p) * 1e6),
                     "form": f"{count} asynchronous calls per direction (one set of kernels per series)",
                     "p50_ms": p(0.5), "p99_ms": p(0.99)},
           "latency_note": "per-series completion time of compression from the start of the pass; "
                           "a batched launch completes every series at its end"}
    out["speedup"] = out["batched"]["gbs"] / out["plain"]["gbs"]
    # every series' stream against the oracle's (threaded driver, host cores)
    from oracle import oracle
    oracle.build()
    t0 = time.perf_counter()
    eq = True
    for x, st in zip(xs, streams):
        eq &= st.cpu().numpy().tobytes() == oracle.compress(x.cpu().numpy(), block, threads=host_cores())
    out["oracle_equal"] = bool(eq)
    out["oracle_check"] = f"all {count} series' streams against the oracle's, {time.perf_counter() - t0:.0f} s"
    comp.close()
    dec.close()
    falcon.set_launch_config(0, 0)
    falcon.set_cta_warps(4, 4)
    return out


def bench_serve(args, dev):
    """Poisson arrivals, 50/50 compress/decompress, request sizes log-uniform 4 KB..256 MB,
    FP64/FP32 50/50, random-walk data (2 places); 64 GB device-memory admission budget.  Each
    offered load is served by the continuous-batching server and, as the baseline, one request
    at a time.  Each load runs for --serve-seconds (shortened from 60 s to keep the bench
    within minutes).  Latency: scheduled arrival -> result seen by the client."""
    from paper_2511_04140_gb300 import serve
    pool = serve.make_pool(count=args.serve_pool, device=dev)
    progress(f"server: pool of {len(pool)} requests built")
    rates = [float(r) for r in args.serve_rates.split(",")]
    window = lambda r: args.serve_seconds if r <= 5000 else args.serve_seconds_saturated
    out = {"workload": f"{len(pool)}-request pool, sizes log-uniform 4 KB..256 MB, FP64/FP32 50/50, "
                       f"50/50 compress/decompress, Poisson arrivals; {args.serve_seconds:g} s per load up to "
                       f"5k req/s, {args.serve_seconds_saturated:g} s above (saturated)",
           "budget_bytes": 64 << 30, "loads": []}
    # the client's Python collector could pause every thread for tens of ms inside a window
    # (this process holds the other sections' objects): collect once, then keep it off while
    # the loads run, for the server and the one-at-a-time baseline alike
    import gc
    gc.collect()
    gc.disable()
    with serve.Server(budget_bytes=64 << 30, host_budget_bytes=16 << 30, device=dev) as srv:
        serve.run_load(srv, pool, rate=500, duration=0.3, seed=99)              # warm-up
        for rate in rates:
            out["loads"].append({"offered_req_s": rate, "seconds": window(rate),
                                 "server": serve.run_load(srv, pool, rate=rate, duration=window(rate),
                                                          seed=int(rate))})
            progress(f"server: {rate:g} req/s done")
        # served results against the oracle: 16 requests of the pool submitted together
        from oracle import oracle
        oracle.build()
        pick = list(range(0, len(pool), max(1, len(pool) // 16)))[:16]
        futs = [srv.submit(*pool[i]) for i in pick]
        eq = True
        for i, f in zip(pick, futs):
            op, payload = pool[i]
            got = f.result().numpy()
            if op == serve.COMPRESS:
                eq &= got.tobytes() == oracle.compress(payload.numpy(), BLOCK, threads=host_cores())
            else:
                want = oracle.decompress(payload.numpy().tobytes(), threads=host_cores())
                eq &= got.tobytes() == want.tobytes()
            del got
        out["oracle_equal"] = bool(eq)
        out["oracle_check"] = f"{len(pick)} pool requests served together, each against the oracle"
    serve.run_one_at_a_time(pool, rate=500, duration=0.3, seed=99, device=dev)   # warm-up
    for ld in out["loads"]:
        rate = ld["offered_req_s"]
        ld["one_at_a_time"] = serve.run_one_at_a_time(pool, rate=rate, duration=window(rate), seed=int(rate),
                                                      device=dev)
        ld["gbs_vs_one_at_a_time"] = ld["server"]["gbs"] / ld["one_at_a_time"]["gbs"]
        progress(f"one at a time: {rate:g} req/s done")
    gc.enable()
    out["client"] = "Python garbage collection off during the timed windows (both forms)"
    return out


def host_link(torch, dev, nbytes=1 << 30):
    """Pinned-memory copy bandwidth in each direction (GB/s), for the end-to-end fractions."""
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    out = {}
    for name, fn in (("h2d", lambda: d.copy_(h, non_blocking=True)), ("d2h", lambda: h.copy_(d, non_blocking=True))):
        fn()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        out[name] = 3 * nbytes / (time.perf_counter() - t0) / 1e9
    return out


def e2e(falcon, torch, bufs, host, dev, args):
    """Same metric through the public host-memory API: the streaming pipeline (H2D ->
    compress -> D2H, then H2D -> decompress -> D2H, 64 MiB frames, 16 streams) on pinned
    buffers; host-to-host time."""
    frame_bytes = 64 << 20
    pinned = {dt: torch.from_numpy(arr).pin_memory() for dt, arr in host.items()}
    outs = {}

    def one():
        h2d = d2h = 0
        for dt, x in pinned.items():
            fv = frame_bytes // x.element_size()
            s, fb = falcon.pipeline_compress(x, block=BLOCK, frame_values=fv, nstreams=16, out=outs.get(dt))
            outs.setdefault(dt, s._base if s._base is not None else s)
            y = falcon.pipeline_decompress(s, fb, nstreams=16)
            h2d += x.numel() * x.element_size() + s.numel()
            d2h += s.numel() + y.numel() * y.element_size()
        return h2d, d2h

    one()
    reps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(reps):
        h2d, d2h = one()
    dt = (time.perf_counter() - t0) / reps
    orig = sum(a.nbytes for a in host.values())
    return {"value": 2 * orig / dt / 1e9, "unit": "GB/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "mode": "falcon_pipeline_compress + falcon_pipeline_decompress, host to host, pinned buffers, "
                    "64 MiB frames, 16 streams", "host_link": host_link(torch, dev)}


def bench_pipeline(falcon, synth, torch, dev, n):
    """2^31 FP64 values (16 GiB) in pinned host memory - random walk with 3 decimal places and
    0.5% full-precision outliers - streamed through the GPU in 64 MiB frames and back."""
    g = torch.Generator(device=dev)
    g.manual_seed(4)
    x = 20.0 + torch.cumsum(torch.randn(n, generator=g, device=dev, dtype=torch.float64) * 0.5, 0)
    vals = torch.round(x * 1000.0) / 1000.0
    mask = torch.rand(n, generator=g, device=dev) < 0.005
    vals = torch.where(mask, x * torch.pow(10.0, torch.rand(n, generator=g, device=dev, dtype=torch.float64) * 5 + 3), vals)
    del x, mask
    t0 = time.perf_counter()
    h = torch.empty(n, dtype=torch.float64, pin_memory=True)
    h.copy_(vals)
    del vals
    torch.cuda.empty_cache()
    out = torch.empty(((n + (1 << 23) - 1) >> 23) * falcon.bound(1 << 23, falcon.F64, BLOCK), dtype=torch.uint8,
                      pin_memory=True)
    back = torch.empty(n, dtype=torch.float64, pin_memory=True)
    setup_s = time.perf_counter() - t0
    # one untimed pass over the whole buffers (the first pass over fresh page-locked memory
    # runs 2-3x slower), then the median of three timed passes per direction
    s, fb = falcon.pipeline_compress(h, block=BLOCK, frame_values=1 << 23, nstreams=16, out=out)
    falcon.pipeline_decompress(s, fb, nstreams=16, out=back)
    tcs, tds = [], []
    for _ in range(3):
        t0 = time.perf_counter()
        s, fb = falcon.pipeline_compress(h, block=BLOCK, frame_values=1 << 23, nstreams=16, out=out)
        tcs.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        y = falcon.pipeline_decompress(s, fb, nstreams=16, out=back)
        tds.append(time.perf_counter() - t0)
    tc, td = statistics.median(tcs), statistics.median(tds)
    ok = bool(torch.equal(y.view(torch.int64), h.view(torch.int64)))
    # frames against the oracle: the first and last two, every 32nd, and the frames around
    # the 4 GiB output offset (64-bit offsets in the host pipeline)
    from oracle import oracle
    oracle.build()
    fv = 1 << 23
    starts = np.concatenate([[0], np.cumsum(np.array(fb, dtype=np.int64))])
    cross = int(np.searchsorted(starts, 1 << 32))
    pick = sorted({0, 1, len(fb) - 2, len(fb) - 1, cross - 2, cross - 1, cross, *range(0, len(fb), 32)} &
                  set(range(len(fb))))
    blob = s.numpy()
    eq = True
    for f in pick:
        part = h[f * fv:(f + 1) * fv].numpy()
        eq &= blob[starts[f]:starts[f + 1]].tobytes() == oracle.compress(part, BLOCK, threads=host_cores())
    link = host_link(torch, dev)
    nbytes = n * 8
    return {"workload": f"{n} FP64 values ({nbytes / 2**30:.1f} GiB) in pinned host memory, random walk, "
                        "3 places, 0.5% outliers; 64 MiB frames, 16 streams",
            "compress_gbs": nbytes / tc / 1e9, "decompress_gbs": nbytes / td / 1e9, "ratio": s.numel() / nbytes,
            "compress_gbs_samples": [round(nbytes / t / 1e9, 1) for t in tcs],
            "decompress_gbs_samples": [round(nbytes / t / 1e9, 1) for t in tds],
            "frames": len(fb), "bit_exact": ok, "host_link_gbs": link, "oracle_equal": bool(eq),
            "oracle_frames": f"{len(pick)} frames: first, last, every 32nd and frames {cross - 2}..{cross} "
                             "around the 4 GiB output offset",
            "compress_frac_of_h2d": nbytes / tc / 1e9 / link["h2d"],
            "decompress_frac_of_d2h": nbytes / td / 1e9 / link["d2h"], "setup_s": setup_s}



# ------------------------------------------------------------------------------ more sections
def time_codec(falcon, torch, x, block, reps=5, variant=0):
    """Kernel times (CUDA events, mean of `reps` after one warm-up) of compressing x with a
    codec variant and decompressing the result, inputs resident; returns the times, the
    stream (device) and whether the round trip is bit-exact."""
    dev = x.device
    code = falcon._dtype_code(x)
    n = x.numel()
    nc = (n + block - 1) // block
    out = torch.empty(max(falcon.variant_bound(n, code, block, variant), 32), dtype=torch.uint8, device=dev)
    ws = torch.zeros(falcon.workspace_bytes(nc), dtype=torch.uint8, device=dev)
    rc = torch.zeros(2, dtype=torch.int64, device=dev)
    rd = torch.zeros(2, dtype=torch.int64, device=dev)
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream(dev)
    falcon.compress_variant_async(x, block, variant, out, ws, rc, stream)
    torch.cuda.synchronize(dev)
    nbytes = int(rc[0].item())
    hdr = out[:32].cpu().numpy().tobytes()
    falcon.decompress_async(out, nbytes, hdr, y, ws, rd, stream)
    torch.cuda.synchronize(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    tc = td = 0.0
    for _ in range(reps):
        ev[0].record(stream)
        falcon.compress_variant_async(x, block, variant, out, ws, rc, stream)
        ev[1].record(stream)
        falcon.decompress_async(out, nbytes, hdr, y, ws, rd, stream)
        ev[2].record(stream)
        torch.cuda.synchronize(dev)
        tc += ev[0].elapsed_time(ev[1])
        td += ev[1].elapsed_time(ev[2])
    iv = torch.int64 if x.dtype == torch.float64 else torch.int32
    ok = int(rc[1].item()) == 0 and int(rd[1].item()) == 0 and torch.equal(y.view(iv), x.view(iv))
    return tc / reps, td / reps, out[:nbytes], bool(ok)


def decimal_segments(n, seed, dtype):
    """The segment workload without outliers and special values: every chunk is Case 1 for
    FP64 (decimals of at most 10 significant digits); FP32 chunks whose decimals exceed 7
    significant digits take Case 2."""
    from paper_2511_04140_gb300 import synth
    return synth.segments(n, seed=seed, dtype=dtype, outlier_rate=0.0, special_rate=0.0)


def bench_case1(falcon, torch, dev, n, peak):
    """Case-1 path at HBM scale: the float-to-integer transform of Eq. 4 (alpha search, exact
    scaling, exact division on decode) on 2^26 values without escapes."""
    out = {"workload": f"decimal segments: {n} values, FP64 and FP32, 4096-value segments with 0..6 "
                       "places, sinusoid + AR(1), no outliers and no special values; block 1024", "kernels": {}}
    for dt in (np.float64, np.float32):
        arr = decimal_segments(n, 7, dt)
        x = torch.from_numpy(arr).to(dev)
        tc, td, st, ok = time_codec(falcon, torch, x, BLOCK, reps=5)
        name = "f64" if dt == np.float64 else "f32"
        nb = st.numel()
        hdr = st[:32 + 4 * ((n + BLOCK - 1) // BLOCK)].cpu().numpy()
        recs = np.frombuffer(st.cpu().numpy().tobytes(), dtype=np.uint8)
        sizes = hdr[32:].view("<u4")
        offs = 32 + 4 * len(sizes) + np.concatenate([[0], np.cumsum(sizes[:-1], dtype=np.int64)])
        alpha = recs[offs]
        case1 = float(np.mean(alpha <= (22 if dt == np.float64 else 10)))
        for kind, ms in (("compress", tc), ("decompress", td)):
            alg = arr.nbytes + nb
            out["kernels"][f"{kind}_{name}"] = {"ms": ms, "gbs_original": arr.nbytes / ms / 1e6,
                                                "hbm_gbs": alg / ms / 1e6, "hbm_frac": alg / ms / 1e6 / peak}
        out[f"ratio_{name}"] = nb / arr.nbytes
        out[f"case1_chunks_{name}"] = case1
        out[f"bit_exact_{name}"] = ok
        del x, st
    torch.cuda.empty_cache()
    return out


def bench_f16(falcon, torch, dev, n, peak):
    """Binary16 (R18) at HBM scale: 2^26 FP16 segment values (128 MiB), per-kernel time, roofline
    fraction, ratio, share of Case-1 chunks; the stream checked against the oracle's on its
    first 4096 chunks and decoded bit-exactly."""
    from oracle import oracle
    from paper_2511_04140_gb300 import synth
    oracle.build()
    arr = synth.segments_f16(n, seed=5)
    x = torch.from_numpy(arr).to(dev)
    tc, td, st, ok = time_codec(falcon, torch, x, BLOCK, reps=5)
    nb = st.numel()
    blob = st.cpu().numpy().tobytes()
    nc = (n + BLOCK - 1) // BLOCK
    sizes = np.frombuffer(blob, dtype="<u4", count=nc, offset=32)
    offs = 32 + 4 * nc + np.concatenate([[0], np.cumsum(sizes[:-1], dtype=np.int64)])
    alpha = np.frombuffer(blob, dtype=np.uint8)[offs]
    out = {"workload": f"FP16 segments: {n} values (128 MiB), 4096-value segments with 0..2 places, amplitude "
                       "10^U(-1,1), sinusoid + AR(1), 0.01% full-precision outliers, 0.001% specials; block 1024",
           "kernels": {}, "ratio": nb / arr.nbytes, "case1_chunks": float(np.mean(alpha <= 4)), "bit_exact": ok,
           "oracle_equal": oracle_equal_sampled(oracle, arr, blob, BLOCK),
           "oracle_check": "the first 4096 chunks' records against the oracle's"}
    for kind, ms in (("compress", tc), ("decompress", td)):
        alg = arr.nbytes + nb
        out["kernels"][f"{kind}_f16"] = {"ms": ms, "gbs_original": arr.nbytes / ms / 1e6, "hbm_gbs": alg / ms / 1e6,
                                         "hbm_frac": alg / ms / 1e6 / peak}
    del x, st
    torch.cuda.empty_cache()
    return out


def bench_analytics(falcon, torch, dev, host, peak):
    """Analytics on compressed data (R19): the aggregate (count, NaN count, min, max, sum) of the
    2^26-value segment streams computed from the records, against decompressing them and
    reducing the values with torch (nanmin/nanmax/nansum-style masked reductions); both timed
    with CUDA events, inputs resident; results compared (count, NaNs, min/max exactly)."""
    out = {"workload": "segment streams of 2^26 values (FP64 and FP32); aggregate = count, NaN count, "
                       "totalOrder min / max and FP64 sum of the non-NaN values", "dtypes": {}}
    stream = torch.cuda.current_stream(dev)
    for dt, name in ((np.float64, "f64"), (np.float32, "f32")):
        x = torch.from_numpy(host[dt]).to(dev)
        s = falcon.compress(x, BLOCK)
        nb = s.numel()
        nc = (x.numel() + BLOCK - 1) // BLOCK
        hdr = s[:32].cpu().numpy().tobytes()
        ws = torch.zeros(falcon.workspace_bytes(nc), dtype=torch.uint8, device=dev)
        st = torch.zeros(falcon.STATS_BYTES, dtype=torch.uint8, device=dev)
        y = torch.empty_like(x)
        rd = torch.zeros(2, dtype=torch.int64, device=dev)

        def agg():
            falcon.aggregate_async(s, nb, hdr, ws, st, stream)

        def dec_reduce():
            falcon.decompress_async(s, nb, hdr, y, ws, rd, stream)
            m = torch.isnan(y)
            v = y.masked_fill(m, 0.0)
            return (m.sum(), v.to(torch.float64).sum(), y.masked_fill(m, float("inf")).min(),
                    y.masked_fill(m, float("-inf")).max())

        times = {}
        for key, fn in (("aggregate", agg), ("decompress_and_reduce", dec_reduce)):
            for _ in range(3):
                fn()
            torch.cuda.synchronize(dev)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ms = []
            for _ in range(10):
                ev[0].record(stream)
                fn()
                ev[1].record(stream)
                torch.cuda.synchronize(dev)
                ms.append(ev[0].elapsed_time(ev[1]))
            times[key] = float(np.median(ms))
        a = falcon.stats_of(st)
        nans, _, vmin, vmax = dec_reduce()
        torch.cuda.synchronize(dev)
        same = (a["status"] == 0 and a["count"] == x.numel() and a["nan_count"] == int(nans)
                and a["min"] == float(vmin) and a["max"] == float(vmax))
        orig = x.numel() * x.element_size()
        out["dtypes"][name] = {
            "aggregate_ms": times["aggregate"], "decompress_and_reduce_ms": times["decompress_and_reduce"],
            "speedup": times["decompress_and_reduce"] / times["aggregate"],
            "aggregate_gbs_original": orig / times["aggregate"] / 1e6,
            "aggregate_hbm_frac": nb / times["aggregate"] / 1e6 / peak,
            "equal_to_decompress_and_reduce": bool(same)}
        del x, s, ws, y
        torch.cuda.empty_cache()
    return out


def oracle_equal_sampled(oracle, vals: np.ndarray, stream: bytes, block: int, chunks: int = 4096, variant: int = 0):
    """The stream's first `chunks` records equal the oracle's records for the same values."""
    nc = (len(vals) + block - 1) // block
    k = min(nc, chunks)
    ref = oracle.compress(vals[:k * block] if k < nc else vals, block, variant=variant, threads=host_cores())
    rec_ref = oracle.chunk_records(ref)
    sizes = np.frombuffer(stream, dtype="<u4", count=nc, offset=32)
    pos = 32 + 4 * nc
    for c in range(k):
        sz = int(sizes[c])
        if stream[pos:pos + sz] != rec_ref[c]:
            return False
        pos += sz
    return True


def bench_variants(falcon, torch, dev, host):
    """The ablation of Sec. 5.4.2 (Fig. 12b): Falcon against Fal._Sparse, Fal._Dense and
    Fal._Elf on the random walk (1,048,576 FP64 values, 2 places) and the segment workload
    (2^26 values, FP64 and FP32): ratio and kernel GB/s per variant; each variant's stream is
    checked against the oracle's on its first 4096 chunks and decoded bit-exactly."""
    from oracle import oracle
    from paper_2511_04140_gb300 import synth
    oracle.build()
    names = {0: "falcon", 1: "fal_sparse", 2: "fal_dense", 3: "fal_elf"}
    works = [("random_walk_f64", synth.random_walk(1 << 20, seed=0, places=2)),
             ("segments_f64", host[np.float64]), ("segments_f32", host[np.float32])]
    out = {"workloads": {}}
    for wname, arr in works:
        x = torch.from_numpy(arr).to(dev)
        rows = {}
        for v, vname in names.items():
            tc, td, st, ok = time_codec(falcon, torch, x, BLOCK, reps=3, variant=v)
            blob = st.cpu().numpy().tobytes()
            rows[vname] = {"ratio": len(blob) / arr.nbytes, "compress_gbs": arr.nbytes / tc / 1e6,
                           "decompress_gbs": arr.nbytes / td / 1e6, "compress_ms": tc, "decompress_ms": td,
                           "bit_exact": ok, "oracle_equal": oracle_equal_sampled(oracle, arr, blob, BLOCK, variant=v)}
        out["workloads"][wname] = rows
        del x
    torch.cuda.empty_cache()
    return out


def bench_schedulers(falcon, torch, dev, n=1 << 28):
    """The scheduler ablation of Sec. 5.4.1 (Fig. 12a): event-driven, sync-based and
    pre-allocation compression of 2 GiB of host values (the host-pipeline generator) in
    64 MiB frames with 1..32 streams; every output equals the event-driven one."""
    g = torch.Generator(device=dev)
    g.manual_seed(6)
    from paper_2511_04140_gb300 import synth
    vals = synth.random_walk_cuda(n, g, places=3, outlier_rate=0.005, device=dev)
    h = torch.empty(n, dtype=torch.float64, pin_memory=True)
    h.copy_(vals)
    del vals
    fv = 1 << 23
    cap = ((n + fv - 1) // fv) * falcon.bound(fv, falcon.F64, BLOCK)
    outs = {sch: torch.empty(cap, dtype=torch.uint8, pin_memory=True) for sch in (0, 1, 2)}
    ref = None
    res = {"workload": f"{n} FP64 values ({n * 8 / 2**30:.0f} GiB) in pinned host memory, random walk, 3 places, "
                       "0.5% outliers; 64 MiB frames", "gbs": {}}
    names = {0: "event_driven", 1: "sync_based", 2: "pre_allocation"}
    ok = True
    for sch, nm in names.items():
        res["gbs"][nm] = {}
        for ns in (1, 2, 4, 8, 16, 32):
            falcon.pipeline_compress(h, block=BLOCK, frame_values=fv, nstreams=ns, out=outs[sch], scheduler=sch)
            t0 = time.perf_counter()
            s, fb = falcon.pipeline_compress(h, block=BLOCK, frame_values=fv, nstreams=ns, out=outs[sch], scheduler=sch)
            dt = time.perf_counter() - t0
            res["gbs"][nm][str(ns)] = n * 8 / dt / 1e9
            if ref is None:
                ref = (s.clone(), fb)
            else:
                ok &= fb == ref[1] and torch.equal(s, ref[0])
    res["bit_exact"] = bool(ok)
    return res


def bench_sweeps(falcon, torch, dev, peak):
    """Parameter sweeps of Sec. 5.3 on synthetic data: decimal places (Fig. 10's beta sweep:
    2^24 FP64 random-walk values rounded to 0..15 places, kernel GB/s and ratio), data size
    (Fig. 11: 100 MB .. 16 GiB through the host pipeline) and frame size (Table 5:
    0.5 .. 8 x 1025 x 1024 values per frame, 2 GiB)."""
    from paper_2511_04140_gb300 import synth
    out = {"places": {}, "data_size": {}, "frame_size": {}}
    g = torch.Generator(device=dev)
    g.manual_seed(8)
    n = 1 << 24
    for pl in range(16):
        x = synth.random_walk_cuda(n, g, places=pl, device=dev)
        tc, td, st, ok = time_codec(falcon, torch, x, BLOCK, reps=3)
        out["places"][str(pl)] = {"ratio": st.numel() / (n * 8), "compress_gbs": n * 8 / tc / 1e6,
                                  "decompress_gbs": n * 8 / td / 1e6, "bit_exact": ok}
    del x
    big = 1 << 31
    vals = synth.random_walk_cuda(big, g, places=3, outlier_rate=0.005, device=dev)
    h = torch.empty(big, dtype=torch.float64, pin_memory=True)
    h.copy_(vals)
    del vals
    torch.cuda.empty_cache()
    fv = 1 << 23
    out_buf = torch.empty(((big + fv - 1) // fv) * falcon.bound(fv, falcon.F64, BLOCK), dtype=torch.uint8,
                          pin_memory=True)
    back = torch.empty(big, dtype=torch.float64, pin_memory=True)
    for mb in (100, 300, 700, 2048, 8192, 16384):
        m = min(big, mb * (1 << 20) // 8)
        part = h[:m]
        falcon.pipeline_compress(part, block=BLOCK, frame_values=fv, out=out_buf)
        t0 = time.perf_counter()
        s, fb = falcon.pipeline_compress(part, block=BLOCK, frame_values=fv, out=out_buf)
        tcp = time.perf_counter() - t0
        falcon.pipeline_decompress(s, fb, out=back)
        t0 = time.perf_counter()
        falcon.pipeline_decompress(s, fb, out=back)
        tdp = time.perf_counter() - t0
        out["data_size"][f"{mb}MB"] = {"compress_gbs": m * 8 / tcp / 1e9, "decompress_gbs": m * 8 / tdp / 1e9}
    part = h[:1 << 28]
    for mult in (0.5, 1, 2, 4, 8):
        fvm = int(mult * 1025 * 1024)
        falcon.pipeline_compress(part, block=BLOCK, frame_values=fvm, out=out_buf)
        t0 = time.perf_counter()
        s, fb = falcon.pipeline_compress(part, block=BLOCK, frame_values=fvm, out=out_buf)
        tcp = time.perf_counter() - t0
        falcon.pipeline_decompress(s, fb, out=back)
        t0 = time.perf_counter()
        falcon.pipeline_decompress(s, fb, out=back)
        tdp = time.perf_counter() - t0
        out["frame_size"][f"{mult}x1025x1024"] = {"compress_gbs": part.numel() * 8 / tcp / 1e9,
                                                  "decompress_gbs": part.numel() * 8 / tdp / 1e9}
    del h, out_buf, back
    return out


if __name__ == "__main__":
    main()
