#!/usr/bin/env python
"""Benchmark of the batched MoA radix-2 FFT on GB300.

Workload (one "step"): the complex128 plain-method configuration at scale,
n = 2^20 with batch 64 (n * batch = 2^26 elements, 1 GiB per buffer), one
forward and one inverse transform of the whole batch.  Inputs are seeded
synthetic data (uniform [-1, 1] real and imaginary parts) resident in HBM;
every buffer is larger than L2 (129 MB), so no flush is needed.

Printed: one JSON line (rank 0) with the metric in GFLOP/s = 5 n log2 n per
transform, the end-to-end figure through host buffers (fft_exec_host), the
roofline of the dominant kernel measured live with CUDA events, the SM
clocks sampled during the timed region, the FP64 CPU oracle timed on a
bounded sample of the same workload, and under "forms" the library's other
configurations measured on the same GPU: the double-float form of the same
step, the complex64 precision forms (FP32, split FP16 / BF16 on the tensor
cores; n = 2^16 x 4096) with their errors against the oracle, the uneven
batch of 20,000 transforms (graph and persistent launch) and forward +
adjoint at n = 2^18 x 256, each with its dominant kernel's roofline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl moafft|reference]
Under torchrun each rank runs the same per-GPU workload on its own GPU
(weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "batched FFT GFLOP/s (5N·log2N) & %HBM roofline, FP64 plain vs FP32/TC at rel err"
UNIT = "GFLOP/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="moafft", choices=["moafft", "reference"])
    ap.add_argument("--log2n", type=int, default=20)
    ap.add_argument("--batch", type=int, default=0, help="override the batch (small profiling cases)")
    ap.add_argument("--e2e-steps", type=int, default=3, help="0 skips the host-buffer measurement")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the other forms (df64, precision, uneven, adjoint)")
    ap.add_argument("--sweep", default="", help="comma-separated log2 n list: extra lines to stderr")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the size sweep (n = 2^12..2^24) the JSON line carries under \"sweep\"")
    ap.add_argument("--case", default="", choices=["", "c1", "c64", "c64_cluster", "c64_rows", "tc_fp16", "tc_bf16", "tc32", "c64_256", "c128", "df64", "dm", "nd2d"],
                    help="small profiling case, three runs: complex64 n=2^16 batch 512 forward "
                         "(c64, tc_*), or complex128 n=2^20 batch 16 forward (c128, df64)")
    ap.add_argument("--extra", action="store_true",
                    help="also measure the other configurations (latency, precision forms, uneven "
                         "batch, forward+adjoint); one JSON line each on stderr")
    return ap.parse_args()


def workload(log2n: int, batch: int = 0):
    n = 1 << log2n
    return n, (batch if batch > 0 else (1 << 26) // n)


def config(n, batch, world):
    return {"workload": f"c128 plain radix-2 FFT, n=2^{int(math.log2(n))}, batch {batch} "
                        f"(n*batch=2^{int(math.log2(n * batch))}, {n * batch * 16 / 2**30:g} GiB per "
                        f"buffer), forward+inverse per step",
            "n": n, "batch_per_gpu": batch, "global_batch": batch * world,
            "dtype": "complex128", "parallelism": f"batch-shard x{world}",
            "l2": "inputs larger than L2 (1 GiB per buffer > 129 MB); no flush"}


def flops_per_step(n, batch):
    return 2 * 5.0 * n * math.log2(n) * batch  # forward + inverse


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi every 200 ms while running: SM clock, its maximum, power
    and the throttle reasons, for the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

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
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- helpers

def code_text(src: str) -> str:
    """A kernel source without its comments and blank space: what the
    traffic record's key tracks (a comment edit leaves the code, and so the
    recorded DRAM traffic, unchanged)."""
    import re
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return " ".join(src.split())


def source_hash() -> str:
    h = hashlib.sha1()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_0803_2386_gb300", "csrc", "*"))):
        with open(f, encoding="utf-8") as fh:
            h.update(os.path.basename(f).encode())
            h.update(code_text(fh.read()).encode())
    return h.hexdigest()[:12]


def recorded_traffic(kernel: str, workload_key: str, transforms=None):
    """DRAM bytes per launch from a committed ncu summary, if it was taken
    on the current kernel sources; else None.  Records taken on a smaller
    batch than the bench's launch hold bytes per transform, scaled here by
    the launch's transforms (the traffic of these passes grows with them)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    e = rec.get(f"{kernel}|{workload_key}")
    if not e or e.get("source_hash") != source_hash():
        return None
    if transforms is not None and "bytes_per_transform" in e:
        return int(round(e["bytes_per_transform"] * transforms))
    return e.get("bytes_per_launch")


def cpu_baseline(n: int, batch: int, target_s: float = 12.0, rows=None):
    """Time the FP64 oracle (as it stands) on the host cores on a bounded
    sample of the workload: forward + inverse of S transforms.  With rows (a
    function s -> (input rows, the GPU's forward spectrum of those rows)),
    the sample is the bench's own first S transforms and the oracle's
    spectrum is also the parity check of the timed GPU output."""
    import numpy as np
    import oracle as O
    import workloads as W
    cores = os.cpu_count() or 1
    x1 = W.uniform_complex(n, 1, seed=0)
    O.lib()  # load (and if needed build) before timing
    t0 = time.perf_counter()
    O.fft(x1, "forward", c=1024, threads=1)
    t1 = max(time.perf_counter() - t0, 1e-3)
    s = int(min(batch, max(cores, math.ceil(target_s / (2 * t1)))))
    s = max(1, min(batch, (s // cores) * cores if s >= cores else s))
    threads = min(cores, s)
    if rows is not None:
        x, Xg = rows(s)
    else:
        x, Xg = W.uniform_complex(n, s, seed=0), None
    t0 = time.perf_counter()
    X = O.fft(x, "forward", c=1024, threads=threads)
    O.fft(X, "inverse", c=1024, threads=threads)
    dt = time.perf_counter() - t0
    gflops = 2 * 5.0 * n * math.log2(n) * s / dt / 1e9
    out = {"value": round(gflops, 4), "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"{s} of the {batch} transforms of n=2^{int(math.log2(n))}, forward+inverse, "
                     f"{threads} threads, {dt:.2f} s wall"}
    # the single-threaded setting: the one forward transform that sized the sample
    out["single_thread"] = {"value": round(5.0 * n * math.log2(n) / t1 / 1e9, 4), "unit": UNIT, "cores": 1,
                            "sample": f"one forward transform of n=2^{int(math.log2(n))}, {t1:.3f} s"}
    if Xg is not None:
        err = np.linalg.norm(Xg - X, axis=-1) / np.linalg.norm(X, axis=-1)
        out["gpu_vs_oracle_rel_err"] = {"transforms": int(s), "max": float(err.max()),
                                        "median": float(np.median(err)), "tolerance": 1e-12}
    return out


# --------------------------------------------------------------- reference

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return 0
    import oracle as O
    import workloads as W
    n, batch = workload(args.log2n, args.batch)
    cores = os.cpu_count() or 1
    s = min(batch, cores)
    x = W.uniform_complex(n, s, seed=0)

    def step():
        X = O.fft(x, "forward", c=1024, threads=s)
        O.fft(X, "inverse", c=1024, threads=s)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    value = 2 * 5.0 * n * math.log2(n) * s / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded uniform[-1,1])",
            "config": config(n, batch, world),
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": s, "kind": "oracle",
                             "sample": f"each step: {s} of the {batch} transforms, forward+inverse, "
                                       f"{s} threads (FP64 CPU oracle, plain C)"},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ moafft

def run_moafft(args):
    import torch
    import paper_0803_2386_gb300 as M
    import workloads as W

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    M.lib()  # no fallback: fails loudly if the library is missing

    n, batch = workload(args.log2n, args.batch)
    x = torch.from_numpy(W.uniform_complex(n, batch, seed=rank)).to(dev)
    X = torch.empty_like(x)
    y = torch.empty_like(x)
    fwd = M.Plan(n, batch, M.FFT_C128, M.FFT_FORWARD)
    inv = M.Plan(n, batch, M.FFT_C128, M.FFT_INVERSE)
    stream = torch.cuda.current_stream(dev)

    def step():
        fwd.exec(x, X, stream)
        inv.exec(X, y, stream)

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize(dev)
    # round-trip check on the warm data (cheap, on device)
    rt = (torch.linalg.vector_norm(y - x) / torch.linalg.vector_norm(x)).item()

    fwd_desc = json.loads(fwd.describe())
    M.fft_plan_profile(fwd.handle, True)
    M.fft_plan_profile(inv.handle, True)
    M.fft_plan_pass_times(fwd.handle)
    M.fft_plan_pass_times(inv.handle)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clocks = sampler.stop()
    t_ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    ms_step = t_ms / args.steps
    value = flops_per_step(n, batch) * world / (ms_step * 1e-3) / 1e9
    launches = args.steps * (fwd.launches + inv.launches)

    # dominant kernel: the pass with the largest accumulated time
    ft = M.fft_plan_pass_times(fwd.handle)
    it = M.fft_plan_pass_times(inv.handle)
    M.fft_plan_profile(fwd.handle, False)
    M.fft_plan_profile(inv.handle, False)
    passes = fwd_desc["schedule"]["passes"]
    per_pass = []
    for i, p in enumerate(passes):
        ms = ft[i][0] + it[i][0]
        cnt = ft[i][1] + it[i][1]
        per_pass.append((ms, cnt, i))
    ms_tot, cnt, dom = max(per_pass)
    chunk = fwd_desc["chunk"]
    log_r = passes[dom]["log_r"]
    avg_ms = ms_tot / max(cnt, 1)
    flops_launch = 5.0 * chunk * n * log_r
    achieved = flops_launch / (avg_ms * 1e-3) / 1e12
    kname = f"tile_kernel<double> pass {dom} (log2 R = {log_r})"
    wkey = f"c128 n=2^{args.log2n}"
    traffic = recorded_traffic(f"pass{dom}", wkey)
    peaks = load_peaks()
    peak64, peak_src = fp64_peak(torch, dev, clocks)
    hbm_step = 2 * 2 * n * batch * 16 / (ms_step * 1e-3) / 1e9
    roofline = {"bound": "alu", "achieved": round(achieved, 4), "peak": round(peak64, 4),
                "unit": "TFLOP/s", "frac": round(achieved / peak64, 4), "traffic": traffic,
                "kernel": kname, "avg_launch_ms": round(avg_ms, 4),
                "algorithmic_per_launch": f"5 flop x {chunk} transforms x 2^{args.log2n} x {log_r} stages",
                "peak_source": peak_src,
                "hbm_gbs_algorithmic_step": round(hbm_step, 1),
                f"hbm_frac_of_{peaks['source']}": round(hbm_step / peaks["hbm_gbs"], 4)}

    e2e = None
    if args.e2e_steps > 0:
        e2e = measure_e2e(M, torch, fwd, inv, x, stream, dev, barrier, dist, n, batch, world, args)
    forms = (measure_forms(M, torch, x, X, stream, n, batch, world, args, dev, clocks, peaks)
             if rank == 0 and not args.no_forms else None)
    sweep = None
    if rank == 0 and not args.no_sweep and args.log2n == 20 and args.batch == 0:
        # the same step across the sizes the configuration sweeps, 2^12..2^24
        sweep = {"config": "c128 FP64, forward + inverse, n * batch = 2^26 (1 GiB per buffer), CUDA events",
                 "points": [sweep_line(M, torch, dev, stream, t, args, quiet=True) for t in range(12, 25, 2)]}

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded uniform[-1,1], seed = rank)",
                "config": config(n, batch, world), "gpu_launches": launches,
                "roundtrip_rel_err": rt, "clocks": clocks, "roofline": roofline, "e2e": e2e,
                "forms": forms, "sweep": sweep}
        if world == 1 and not args.no_cpu_baseline:
            fwd.exec(x, X, stream)  # the timed forward spectrum (deterministic)
            torch.cuda.synchronize()
            line["cpu_baseline"] = cpu_baseline(
                n, batch, rows=lambda s: (x[:s].cpu().numpy(), X[:s].cpu().numpy()))
        print(json.dumps(line), flush=True)

    for t in [int(v) for v in args.sweep.split(",") if v.strip()]:
        sweep_line(M, torch, dev, stream, t, args)
    if args.extra and rank == 0:
        extra_configs(M, torch, dev, stream)

    fwd.close()
    inv.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def load_peaks():
    """Roofline denominators: MEASURED_PEAKS.json (written on this GPU pool:
    a STREAM-style copy and a cuBLAS bf16 GEMM) when present, else one
    earlier GB300 measurement (6.8 TB/s, 1.9 PFLOP/s bf16) marked as a
    fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
        return {"hbm_gbs": float(peaks["hbm_gbs"]), "bf16_tflops": float(peaks.get("bf16_tflops", 1900.0)),
                "source": "measured"}
    except (OSError, ValueError, KeyError, TypeError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


def fp64_peak(torch, dev, clocks):
    """FP64 issue peak of this GPU: SMs (from the device) x 2 DFMA per SM per
    clock (GB300's FP64 unit count, its nominal 1.25 TFLOP/s) x 2 flop x the
    maximum SM clock (nvidia-smi, sampled with the timed region; 2070 MHz if
    it could not be read).  A probe of independent FP64 chains sustains 84 %
    of this (1.68 operations per SM per clock); FMA-only code keeps the
    FP64 pipe up to about 90 % busy."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    return sms * 2 * 2 * mhz * 1e6 / 1e12, (f"FP64 issue peak: {sms} SMs x 2 DFMA/clk x 2 flop x {mhz:g} MHz "
                                             "(SM count from the device, maximum SM clock from nvidia-smi)")


def profiled(M, torch, stream, handles, fn, reps):
    """Run fn reps times with the plans' launch timing on and return, for
    the pass with the largest accumulated time over the plans in `handles`,
    (plan index, pass index, launches, average ms per launch)."""
    for h in handles:
        M.fft_plan_profile(h, True)
        M.fft_plan_pass_times(h)
    for _ in range(reps):
        fn()
    torch.cuda.synchronize()
    best = None
    for k, h in enumerate(handles):
        for i, (ms, cnt) in enumerate(M.fft_plan_pass_times(h)):
            if cnt and (best is None or ms > best[0]):
                best = (ms, k, i, cnt)
        M.fft_plan_profile(h, False)
    ms, k, i, cnt = best
    return k, i, cnt, ms / cnt


def hbm_roofline(kernel, bytes_per_launch, avg_ms, peaks, what, traffic=None):
    """Roofline record of an HBM-bound kernel: algorithmic bytes per launch
    over its average launch time, against the HBM copy peak; traffic: the
    recorded DRAM bytes per launch, when there is a record."""
    gbs = bytes_per_launch / (avg_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": round(gbs, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": round(gbs / peaks["hbm_gbs"], 4), "traffic": traffic, "kernel": kernel,
            "avg_launch_ms": round(avg_ms, 4), "algorithmic_per_launch": what,
            "peak_source": f"HBM copy peak ({peaks['source']})"}


def oracle_rows_err(O, np, got_rows, in_rows, op):
    """Parity error of sampled transforms against the FP64 oracle: per row,
    the larger of the relative L2 error and the largest element error over
    the largest element."""
    ref = O.fft(np.asarray(in_rows, dtype=np.complex128), op, c=1024, threads=max(1, len(in_rows)))
    d = np.asarray(got_rows, dtype=np.complex128) - ref
    e2 = np.linalg.norm(d, axis=-1) / np.linalg.norm(ref, axis=-1)
    ei = np.abs(d).max(axis=-1) / np.abs(ref).max(axis=-1)
    return float(np.maximum(e2, ei).max())


def measure_forms(M, torch, x, X, stream, n, batch, world, args, dev, clocks, peaks):
    """The library's other forms, each timed on this GPU with its dominant
    kernel's roofline (measured with CUDA events around every launch, as the
    headline's):
      df64        the headline step in double-float butterflies (FP32 pipes),
                  with its error against the FP64 path and against the FP64
                  oracle on three sampled transforms;
      fp32, tc_fp16, tc_bf16
                  complex64 n = 2^16, batch 4096, forward (the precision
                  configuration), Gaussian sigma = 1 input, with the error
                  against the FP64 oracle on sampled transforms for that
                  input and for amplitudes 10^U(-4, 4); speed-up over the
                  FP64 path on the same transforms;
      uneven      20,000 complex64 transforms of 2^6..2^16 points (sizes from
                  default_rng(1)) as the default graph and as one persistent
                  launch;
      fwd_adjoint complex64 n = 2^18, batch 256: forward + adjoint (the
                  differentiation configuration's two transforms)."""
    import numpy as np
    import oracle as O
    import workloads as W
    reps = max(3, args.steps // 2)
    forms = {}
    # ---- double-float form of the headline step
    if n >= 16:
        y = torch.empty_like(x)
        r = torch.empty_like(x)
        pf = M.Plan(n, batch, M.FFT_C128, M.FFT_FORWARD, M.FFT_FORM_DF64)
        pi = M.Plan(n, batch, M.FFT_C128, M.FFT_INVERSE, M.FFT_FORM_DF64)

        def step():
            pf.exec(x, y, stream)
            pi.exec(y, r, stream)

        ms = _time(torch, stream, step, reps, warm=2)
        err = (torch.linalg.vector_norm((y - X).flatten()) / torch.linalg.vector_norm(X.flatten())).item()
        # three sampled transforms against the FP64 oracle (y: the timed forward output)
        dpicks = [0, batch // 2, batch - 1]
        err_oracle = oracle_rows_err(O, np, y[dpicks].cpu().numpy(), x[dpicks].cpu().numpy(), "forward")
        k, i, cnt, avg = profiled(M, torch, stream, [pf.handle, pi.handle], step, 2)
        desc = json.loads((pf if k == 0 else pi).describe())
        lr = desc["schedule"]["passes"][i]["log_r"]
        chunk = desc["chunk"]
        fl = 5.0 * chunk * n * lr
        forms["df64"] = {"value": round(flops_per_step(n, batch) * world / (ms * 1e-3) / 1e9, 3), "unit": UNIT,
                         "ms_per_step": round(ms, 4), "dtype": "f32x2 (double-float)",
                         "rel_err_vs_fp64_path": err,
                         "rel_err_vs_oracle": {"max": err_oracle, "transforms": len(dpicks)}, "tolerance": 1e-12,
                         "roofline": {"bound": "alu", "achieved": round(fl / (avg * 1e-3) / 1e12, 4),
                                      "unit": "TFLOP/s", "kernel": f"tile_kernel<dfloat> pass {i} (log2 R = {lr})",
                                      "avg_launch_ms": round(avg, 4),
                                      "algorithmic_per_launch": f"5 flop x {chunk} transforms x 2^{int(math.log2(n))} x {lr} stages",
                                      "traffic": recorded_traffic(f"df64 pass{i}", f"c128 n=2^{int(math.log2(n))}",
                                                                  transforms=chunk),
                                      "note": "FP32 issue-bound; no FP64 instruction"}}
        pf.close()
        pi.close()
        del y, r
    # ---- precision forms at complex64 n = 2^16, batch 4096
    n3, b3 = 1 << 16, 4096
    g = torch.Generator(device=dev).manual_seed(0)
    xg = torch.randn(b3, n3, dtype=torch.complex64, device=dev, generator=g)
    u = torch.rand(2, b3, n3, dtype=torch.float32, device=dev, generator=torch.Generator(device=dev).manual_seed(0))
    amp = torch.pow(10.0, 8.0 * u[0] - 4.0)
    xd = torch.polar(amp, 2.0 * math.pi * u[1])
    del u, amp
    yo = torch.empty_like(xg)
    x128 = xg.to(torch.complex128)
    y128 = torch.empty_like(x128)
    p64 = M.Plan(n3, b3, M.FFT_C128, M.FFT_FORWARD)
    ms64 = _time(torch, stream, lambda: p64.exec(x128, y128, stream), max(2, reps // 2))
    p64.close()
    del x128, y128
    fl3 = 5.0 * n3 * 16 * b3
    picks = [0, 2049, b3 - 1]
    xg_rows = xg[picks].cpu().numpy()
    xd_rows = xd[picks].cpu().numpy()
    for form, name in ((M.FFT_FORM_PLAIN, "fp32"), (M.FFT_FORM_TC_FP16, "tc_fp16"), (M.FFT_FORM_TC_BF16, "tc_bf16")):
        pf = M.Plan(n3, b3, M.FFT_C64, M.FFT_FORWARD, form)
        ms = _time(torch, stream, lambda: pf.exec(xg, yo, stream), reps)
        M.fft_plan_check(pf.handle)
        eg = oracle_rows_err(O, np, yo[picks].cpu().numpy(), xg_rows, "forward")
        _, i, cnt, avg = profiled(M, torch, stream, [pf.handle], lambda: pf.exec(xg, yo, stream), 2)
        desc = json.loads(pf.describe())
        chunk = desc["chunk"]
        lr = desc["schedule"]["passes"][i]["log_r"]
        pf.exec(xd, yo, stream)
        torch.cuda.synchronize()
        M.fft_plan_check(pf.handle)
        ed = oracle_rows_err(O, np, yo[picks].cpu().numpy(), xd_rows, "forward")
        gbs = 2 * n3 * b3 * 8 / (ms * 1e-3) / 1e9
        kname = {"fp32": "bulk_kernel", "tc_fp16": "tc kernel (split FP16)", "tc_bf16": "tc kernel (split BF16)"}[name]
        forms[name] = {"config": "c64 n=2^16 batch 4096 forward", "value": round(fl3 / (ms * 1e-3) / 1e9, 1),
                       "unit": UNIT, "ms": round(ms, 4), "gbs_algorithmic": round(gbs, 1),
                       f"hbm_frac_of_{peaks['source']}": round(gbs / peaks["hbm_gbs"], 4),
                       "passes": len(desc["schedule"]["passes"]),
                       "rel_err_vs_oracle": {"gaussian": eg, "dynamic_range_1e-4_1e4": ed,
                                             "transforms": len(picks)},
                       "tolerance": 1e-6 * 16 if form == M.FFT_FORM_PLAIN else 1e-5 * 16,
                       "speedup_vs_fp64": round(ms64 / ms, 2), "fp64_ms": round(ms64, 4),
                       "roofline": hbm_roofline(f"{kname} pass {i} (log2 R = {lr})", 2 * chunk * n3 * 8, avg, peaks,
                                                f"one read + one write of {chunk} transforms x 2^16 x 8 B",
                                                recorded_traffic(f"{name} pass{i}", "c64 n=2^16", transforms=chunk))}
        pf.close()
    del xg, xd, yo
    # ---- uneven batch: 20,000 transforms of 2^6..2^16 points
    sizes, _ = W.uneven_sizes()
    total = int(sizes.sum())
    xu = (torch.rand(total, dtype=torch.complex64, device=dev, generator=torch.Generator(device=dev).manual_seed(1))
          * 2 - (1 + 1j))
    yu = torch.empty_like(xu)
    flu = float(np.sum(5.0 * sizes * np.log2(sizes)))
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    pick = [0, len(sizes) // 2, len(sizes) - 1]
    row = {"config": "c64 uneven batch, 20000 transforms, n = 2^6..2^16 (default_rng(1))", "points": total}
    for label, env in (("graph", None), ("persistent", "1")):
        if env:
            os.environ["MOAFFT_PERSIST"] = env
        pm = M.fft_plan_many(sizes, M.FFT_C64, M.FFT_FORWARD)
        if env:
            del os.environ["MOAFFT_PERSIST"]
        ms = _time(torch, stream, lambda: M.fft_exec(pm, xu, yu, stream), reps)
        M.fft_plan_check(pm)
        errs = []
        for t in pick:
            o, s_ = int(offs[t]), int(sizes[t])
            errs.append(oracle_rows_err(O, np, yu[o:o + s_].cpu().numpy()[None], xu[o:o + s_].cpu().numpy()[None],
                                        "forward"))
        gbs = 2 * total * 8 / (ms * 1e-3) / 1e9
        row[label] = {"ms": round(ms, 4), "value": round(flu / (ms * 1e-3) / 1e9, 1), "unit": UNIT,
                      "launches": M.fft_plan_launches(pm), "gbs_one_round_trip": round(gbs, 1),
                      f"hbm_frac_of_{peaks['source']}": round(gbs / peaks["hbm_gbs"], 4),
                      "rel_err_vs_oracle": max(errs)}
        M.fft_destroy(pm)
    row["tolerance"] = 1e-6 * 16
    forms["uneven"] = row
    del xu, yu
    # ---- forward + adjoint, complex64 n = 2^18, batch 256
    n5, b5 = 1 << 18, 256
    x5 = (torch.rand(b5, n5, dtype=torch.complex64, device=dev, generator=torch.Generator(device=dev).manual_seed(0))
          * 2 - (1 + 1j))
    y5 = torch.empty_like(x5)
    g5 = torch.empty_like(x5)
    pd = M.Plan(n5, b5, M.FFT_C64, M.FFT_FORWARD)

    def fwd_adj():
        pd.exec(x5, y5, stream)
        pd.exec_adjoint(y5, g5, stream)

    ms = _time(torch, stream, fwd_adj, reps)
    ea = oracle_rows_err(O, np, g5[:2].cpu().numpy(), y5[:2].cpu().numpy(), "adjoint_forward")
    _, i, cnt, avg = profiled(M, torch, stream, [pd.handle], fwd_adj, 2)
    desc = json.loads(pd.describe())
    chunk = desc["chunk"]
    lr = desc["schedule"]["passes"][i]["log_r"]
    gbs = 2 * 2 * n5 * b5 * 8 / (ms * 1e-3) / 1e9
    forms["fwd_adjoint"] = {"config": "c64 n=2^18 batch 256, forward + adjoint", "ms": round(ms, 4),
                            "value": round(2 * 5.0 * n5 * 18 * b5 / (ms * 1e-3) / 1e9, 1), "unit": UNIT,
                            "gbs_algorithmic": round(gbs, 1),
                            f"hbm_frac_of_{peaks['source']}": round(gbs / peaks["hbm_gbs"], 4),
                            "adjoint_rel_err_vs_oracle": ea, "tolerance": 1e-6 * 18,
                            "roofline": hbm_roofline(f"bulk_kernel pass {i} (log2 R = {lr})", 2 * chunk * n5 * 8, avg,
                                                     peaks, f"one read + one write of {chunk} transforms x 2^18 x 8 B")}
    pd.close()
    del x5, y5, g5
    torch.cuda.empty_cache()
    return forms


def measure_e2e(M, torch, fwd, inv, x, stream, dev, barrier, dist, n, batch, world, args):
    """End to end through host buffers (pinned): H2D and D2H inside the timing."""
    xh = x.cpu().pin_memory()
    Xh = torch.empty_like(xh).pin_memory()
    yh = torch.empty_like(xh).pin_memory()

    def e2e_step():
        M.fft_exec_host(fwd.handle, xh, Xh, stream)
        M.fft_exec_host(inv.handle, Xh, yh, stream)

    e2e_step()
    torch.cuda.synchronize(dev)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        e2e_step()
    torch.cuda.synchronize(dev)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps, dist, dev)
    rt_host = float((torch.linalg.vector_norm(yh - xh) / torch.linalg.vector_norm(xh)).item())
    bytes_buf = n * batch * 16
    e2e = {"value": round(flops_per_step(n, batch) * world / e2e_s / 1e9, 3), "unit": UNIT,
           "h2d_bytes_per_step": 2 * bytes_buf, "d2h_bytes_per_step": 2 * bytes_buf,
           "ms_per_step": round(e2e_s * 1e3, 3), "api": "fft_exec_host (pinned host buffers)",
           "roundtrip_rel_err": rt_host}
    return e2e


def sweep_line(M, torch, dev, stream, log2n, args, quiet=False):
    """The headline step (complex128 FP64, forward + inverse, n * batch =
    2^26) at n = 2^log2n: GFLOP/s from CUDA events over max(1, steps / 2)
    steps after two warm-up steps, and the round-trip error."""
    n, batch = workload(log2n)
    gen = torch.Generator(device=dev).manual_seed(log2n)
    x = torch.rand(batch, n, dtype=torch.complex128, device=dev, generator=gen) * 2 - (1 + 1j)
    X = torch.empty_like(x)
    y = torch.empty_like(x)
    fwd = M.Plan(n, batch, M.FFT_C128, M.FFT_FORWARD)
    inv = M.Plan(n, batch, M.FFT_C128, M.FFT_INVERSE)
    for _ in range(2):
        fwd.exec(x, X, stream)
        inv.exec(X, y, stream)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    k = max(1, args.steps // 2)
    for _ in range(k):
        fwd.exec(x, X, stream)
        inv.exec(X, y, stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / k
    rt = (torch.linalg.vector_norm((y - x).flatten()) / torch.linalg.vector_norm(x.flatten())).item()
    row = {"n": n, "batch": batch, "ms_per_step": round(ms, 4),
           "gflops": round(flops_per_step(n, batch) / (ms * 1e-3) / 1e9, 2), "roundtrip_rel_err": rt}
    if not quiet:
        print(json.dumps(dict(sweep=True, **row)), file=sys.stderr, flush=True)
    fwd.close()
    inv.close()
    return row


def _time(torch, stream, fn, reps, warm=2):
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _emit(d):
    print(json.dumps(d), file=sys.stderr, flush=True)


def extra_configs(M, torch, dev, stream):
    """The remaining configurations, measured on the same GPU.  Errors are
    relative L2 against the library's own FP64 (complex128) path, which the
    test-suite checks against the oracle."""
    import numpy as np
    import workloads as W
    torch.manual_seed(0)  # every synthetic input below is seeded
    peaks = load_peaks()
    hbm = peaks["hbm_gbs"]
    frac_key = f"hbm_frac_of_{peaks['source']}"

    def rel(a, b):
        return (torch.linalg.vector_norm((a.to(torch.complex128) - b).flatten()) /
                torch.linalg.vector_norm(b.flatten())).item()

    # latency: complex128 n = 2^10, batch 1
    n = 1 << 10
    x = torch.from_numpy(W.uniform_complex(n, 1, seed=0)).to(dev)
    y = torch.empty_like(x)
    p = M.Plan(n, 1, M.FFT_C128, M.FFT_FORWARD)
    ms = _time(torch, stream, lambda: p.exec(x, y, stream), 200)
    # device time per call without the host: 50 calls captured in one CUDA
    # graph, replayed between events
    # (graphs are captured on a side stream)
    graph = torch.cuda.CUDAGraph()
    cs = torch.cuda.Stream(device=dev)
    cs.wait_stream(torch.cuda.current_stream(dev))
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(cs):
        with torch.cuda.graph(graph, stream=cs):
            for _ in range(50):
                p.exec(x, y, cs)
        graph.replay()
        cs.synchronize()
        e0.record(cs)
        graph.replay()
        e1.record(cs)
        cs.synchronize()
    kms = e0.elapsed_time(e1) / 50
    ref = torch.fft.fft(x.to(torch.complex128))
    _emit({"config": "c128 n=2^10 batch 1 forward", "schedule": [q["log_r"] for q in json.loads(p.describe())["schedule"]["passes"]],
           "us_per_call_host_bound": round(ms * 1e3, 3),
           "us_per_call_device": round(kms * 1e3, 3), "gflops_device": round(5 * n * 10 / (kms * 1e-3) / 1e9, 3),
           "rel_err_vs_torch_fft": rel(y, ref)})
    p.close()

    # precision forms: complex64 n = 2^16, batch 4096 (Gaussian sigma = 1)
    n, batch = 1 << 16, 4096
    xc = torch.randn(batch, n, dtype=torch.complex64, device=dev, generator=torch.Generator(dev).manual_seed(0))
    ref = torch.empty(batch, n, dtype=torch.complex128, device=dev)
    p64 = M.Plan(n, batch, M.FFT_C128, M.FFT_FORWARD)
    x128 = xc.to(torch.complex128)
    ms64 = _time(torch, stream, lambda: p64.exec(x128, ref, stream), 3)
    del x128
    p64.close()
    fl = 5.0 * n * 16 * batch
    _emit({"config": "c128 FP64 plain n=2^16 batch 4096 forward", "ms": round(ms64, 3),
           "gflops": round(fl / (ms64 * 1e-3) / 1e9, 1)})
    out = torch.empty_like(xc)
    for form, name in ((M.FFT_FORM_PLAIN, "FP32 plain"), (M.FFT_FORM_TC_FP16, "TC split FP16"),
                       (M.FFT_FORM_TC_BF16, "TC split BF16")):
        pf = M.Plan(n, batch, M.FFT_C64, M.FFT_FORWARD, form)
        ms = _time(torch, stream, lambda: pf.exec(xc, out, stream), 5)
        M.fft_plan_check(pf.handle)
        gbs = 2 * n * batch * 8 / (ms * 1e-3) / 1e9
        _emit({"config": f"c64 {name} n=2^16 batch 4096 forward", "ms": round(ms, 3),
               "gflops": round(fl / (ms * 1e-3) / 1e9, 1), "gbs": round(gbs, 1),
               frac_key: round(gbs / hbm, 4),
               "rel_err_vs_fp64": rel(out, ref), "speedup_vs_fp64": round(ms64 / ms, 2),
               "tolerance": 1e-6 * 16 if form == M.FFT_FORM_PLAIN else 1e-5 * 16})
        pf.close()
    del ref, out, xc
    # the same forms on the dynamic-range input (amplitudes 10^U(-4, 4), seed 0)
    nb = 256
    xd = torch.from_numpy(W.dynamic_range_complex(n, nb, seed=0)).to(dev)
    refd = torch.empty_like(xd)
    p64 = M.Plan(n, nb, M.FFT_C128, M.FFT_FORWARD)
    p64.exec(xd.to(torch.complex64).to(torch.complex128), refd, stream)
    p64.close()
    xd64 = xd.to(torch.complex64)
    outd = torch.empty_like(xd64)
    row = {"config": f"c64 precision forms, dynamic range 1e-4..1e4, n=2^16 batch {nb} forward (error vs FP64 path)"}
    for form, name in ((M.FFT_FORM_PLAIN, "fp32"), (M.FFT_FORM_TC_FP16, "tc_fp16"), (M.FFT_FORM_TC_BF16, "tc_bf16")):
        pf = M.Plan(n, nb, M.FFT_C64, M.FFT_FORWARD, form)
        pf.exec(xd64, outd, stream)
        torch.cuda.synchronize()
        M.fft_plan_check(pf.handle)
        row[f"{name}_rel_err"] = rel(outd, refd)
        pf.close()
    row["tolerance_fp32"] = 1e-6 * 16
    row["tolerance_tc"] = 1e-5 * 16
    _emit(row)
    del xd, refd, xd64, outd

    # uneven batch: 20,000 complex64 transforms, n in 2^6..2^16 (seed 1)
    sizes, data = W.uneven_batch()
    xu = torch.from_numpy(data).to(torch.complex64).to(dev)
    yu = torch.empty_like(xu)
    os.environ["MOAFFT_PERSIST"] = "1"
    pm = M.fft_plan_many(sizes, M.FFT_C64, M.FFT_FORWARD)
    del os.environ["MOAFFT_PERSIST"]
    ms_pers = _time(torch, stream, lambda: M.fft_exec(pm, xu, yu, stream), 10)
    M.fft_plan_check(pm)
    pers = json.loads(M.fft_plan_describe(pm))["persistent"]
    M.fft_destroy(pm)
    pm = M.fft_plan_many(sizes, M.FFT_C64, M.FFT_FORWARD)
    ms_g = _time(torch, stream, lambda: M.fft_exec(pm, xu, yu, stream), 10)
    launches = M.fft_plan_launches(pm)
    M.fft_destroy(pm)
    # the same plan after the autotuner has timed every candidate schedule of
    # each length at its count (a fresh cache file, so nothing is reused)
    import tempfile
    old_cache = os.environ.get("MOAFFT_TUNE_CACHE")
    with tempfile.TemporaryDirectory() as tdir:
        os.environ["MOAFFT_TUNE_CACHE"] = os.path.join(tdir, "tune.jsonl")
        t_tune = time.perf_counter()
        lengths, counts = np.unique(sizes, return_counts=True)
        for s_, c_ in zip(lengths.tolist(), counts.tolist()):
            M.Plan(int(s_), int(c_), M.FFT_C64, M.FFT_FORWARD, M.FFT_FORM_PLAIN, "auto").close()
        tune_s = time.perf_counter() - t_tune
        pm = M.fft_plan_many(sizes, M.FFT_C64, M.FFT_FORWARD)
        ms_t = _time(torch, stream, lambda: M.fft_exec(pm, xu, yu, stream), 10)
        M.fft_plan_check(pm)
        M.fft_destroy(pm)
    if old_cache is None:
        del os.environ["MOAFFT_TUNE_CACHE"]
    else:
        os.environ["MOAFFT_TUNE_CACHE"] = old_cache
    plans = {}
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]])

    def per_transform():
        for s_, o in zip(sizes.tolist(), offs.tolist()):
            if s_ not in plans:
                plans[s_] = M.fft_plan(s_, 1, M.FFT_C64, M.FFT_FORWARD)
            M.fft_exec(plans[s_], xu[o:o + s_], yu[o:o + s_], stream)

    ms_p = _time(torch, stream, per_transform, 1, warm=1)
    for h in plans.values():
        M.fft_destroy(h)
    fl = float(sum(5 * s_ * np.log2(s_) for s_ in sizes.tolist()))
    _emit({"config": "c64 uneven batch 20000 transforms n=2^6..2^16",
           "persistent_ms": round(ms_pers, 3), "persistent": pers,
           "persistent_gflops": round(fl / (ms_pers * 1e-3) / 1e9, 1), "graph_ms": round(ms_g, 3),
           "graph_launches": launches, "graph_gflops": round(fl / (ms_g * 1e-3) / 1e9, 1),
           "graph_autotuned_ms": round(ms_t, 3), "autotune_s": round(tune_s, 1),
           "per_transform_launch_ms": round(ms_p, 3), "speedup": round(ms_p / ms_g, 1)})
    del xu, yu

    # complex128 at FP64 accuracy: native FP64 vs double-float butterflies
    n, batch = 1 << 20, 64
    xd = torch.rand(batch, n, dtype=torch.complex128, device=dev) * 2 - (1 + 1j)
    yd = torch.empty_like(xd)
    rd = torch.empty_like(xd)
    res = {}
    for form, name in ((M.FFT_FORM_PLAIN, "fp64"), (M.FFT_FORM_DF64, "df64")):
        pf = M.Plan(n, batch, M.FFT_C128, M.FFT_FORWARD, form)
        pi = M.Plan(n, batch, M.FFT_C128, M.FFT_INVERSE, form)

        def fwd_inv():
            pf.exec(xd, yd, stream)
            pi.exec(yd, rd, stream)

        res[name] = _time(torch, stream, fwd_inv, 5)
        if name == "fp64":
            ref = yd.clone()
        else:
            res["df64_err"] = rel(yd, ref)
        res[name + "_rt"] = rel(rd, xd)
        pf.close()
        pi.close()
    fl = 2 * 5.0 * n * 20 * batch
    _emit({"config": "c128 n=2^20 batch 64 forward+inverse: FP64 vs double-float",
           "fp64_ms": round(res["fp64"], 3), "fp64_gflops": round(fl / (res["fp64"] * 1e-3) / 1e9, 1),
           "df64_ms": round(res["df64"], 3), "df64_gflops": round(fl / (res["df64"] * 1e-3) / 1e9, 1),
           "df64_rel_err_vs_fp64": res["df64_err"], "df64_roundtrip_err": res["df64_rt"],
           "speedup": round(res["fp64"] / res["df64"], 2)})
    del xd, yd, rd, ref

    # cache-blocked passes vs the unblocked routine (one HBM pass per stage)
    for dtn, nn_, bb_, tdt in ((M.FFT_C64, 1 << 16, 4096, torch.complex64),
                               (M.FFT_C128, 1 << 20, 64, torch.complex128)):
        xa = torch.randn(bb_, nn_, dtype=tdt, device=dev, generator=torch.Generator(dev).manual_seed(6))
        ya = torch.empty_like(xa)
        res = {}
        for sched in (None, "stages", "stages_stride"):
            pa = M.Plan(nn_, bb_, dtn, M.FFT_FORWARD, M.FFT_FORM_PLAIN, sched)
            res[sched or "passes"] = _time(torch, stream, lambda: pa.exec(xa, ya, stream), 3)
            res[(sched or "passes") + "_launches"] = pa.launches
            pa.close()
        fl = 5.0 * nn_ * math.log2(nn_) * bb_
        _emit({"config": f"{'c64' if dtn == M.FFT_C64 else 'c128'} n=2^{int(math.log2(nn_))} batch {bb_} "
                         "forward: blocked passes vs one pass per stage",
               "blocked_ms": round(res["passes"], 3), "blocked_launches": res["passes_launches"],
               "per_stage_ms": round(res["stages"], 3), "per_stage_launches": res["stages_launches"],
               "blocked_gflops": round(fl / (res["passes"] * 1e-3) / 1e9, 1),
               "per_stage_gflops": round(fl / (res["stages"] * 1e-3) / 1e9, 1),
               "per_stage_stride_order_ms": round(res["stages_stride"], 3),
               "speedup": round(res["stages"] / res["passes"], 2)})
        del xa, ya

    # differentiation: complex64 n = 2^18, batch 256, forward + adjoint
    n, batch = 1 << 18, 256
    xd = torch.randn(batch, n, dtype=torch.complex64, device=dev)
    yd = torch.empty_like(xd)
    gd = torch.empty_like(xd)
    pd = M.Plan(n, batch, M.FFT_C64, M.FFT_FORWARD)

    def fwd_adj():
        pd.exec(xd, yd, stream)
        pd.exec_adjoint(yd, gd, stream)

    ms = _time(torch, stream, fwd_adj, 5)
    _emit({"config": "c64 n=2^18 batch 256 forward + adjoint", "ms": round(ms, 3),
           "gflops": round(2 * 5.0 * n * 18 * batch / (ms * 1e-3) / 1e9, 1),
           "gbs": round(4 * n * batch * 8 / (ms * 1e-3) / 1e9, 1)})
    pd.close()

    # multi-dimensional transforms (the last axis as 1-D transforms, each
    # other axis one column pass); error against the complex128 plan on the
    # same input (the parity tests check that one against the oracle)
    for dims, batch, f64 in (((4096, 4096), 8, False), ((256, 256, 256), 8, False),
                             ((2048, 2048), 16, True), ((128, 128, 128), 32, True)):
        npts = math.prod(dims)
        tdt = torch.complex128 if f64 else torch.complex64
        gen = torch.Generator(device=dev).manual_seed(len(dims))
        x = torch.randn((batch,) + dims, dtype=tdt, device=dev, generator=gen)
        y = torch.empty_like(x)
        pn = M.PlanND(dims, batch, M.FFT_C128 if f64 else M.FFT_C64, M.FFT_FORWARD)
        ms = _time(torch, stream, lambda: pn.exec(x, y, stream), 5)
        row = {"config": f"{'c128' if f64 else 'c64'} {len(dims)}-D {'x'.join(map(str, dims))} batch {batch} forward",
               "ms": round(ms, 3), "launches": pn.launches,
               "gflops": round(5.0 * npts * math.log2(npts) * batch / (ms * 1e-3) / 1e9, 1),
               "gbs_one_round_trip": round(2 * npts * batch * (16 if f64 else 8) / (ms * 1e-3) / 1e9, 1)}
        if not f64:
            xr = x[:1].to(torch.complex128)
            yr = torch.empty_like(xr)
            with M.PlanND(dims, 1, M.FFT_C128, M.FFT_FORWARD) as pr:
                pr.exec(xr, yr, stream)
            row["rel_err_vs_fp64"] = rel(y[:1], yr)
        _emit(row)
        pn.close()
        del x, y

    # radix sweep at n = 2^24 (the paper's Table 4 sweeps the radix of
    # fftpsiradn at 2^24): three passes of 2^8 through the generic tile kernel
    # (width 8 keeps every variant on the same kernel), register digits of
    # 2, 4, 8 and 16 points; the default schedule beside them
    for f64, batch in ((False, 8), (True, 4)):
        n = 1 << 24
        tdt = torch.complex128 if f64 else torch.complex64
        gen = torch.Generator(device=dev).manual_seed(24)
        x = torch.randn(batch, n, dtype=tdt, device=dev, generator=gen)
        y = torch.empty_like(x)
        row = {"config": f"radix sweep, {'c128' if f64 else 'c64'} n=2^24 batch {batch} forward"}
        for k in (1, 2, 3, 4, None):
            sched = None if k is None else f"8@8/{k},8@8/{k},8@8/{k}"
            p = M.Plan(n, batch, M.FFT_C128 if f64 else M.FFT_C64, M.FFT_FORWARD, M.FFT_FORM_PLAIN, sched)
            ms = _time(torch, stream, lambda: p.exec(x, y, stream), 3)
            key = "default_ms" if k is None else f"radix{1 << k}_ms"
            row[key] = round(ms, 3)
            p.close()
        _emit(row)
        del x, y

    # tensor-core DFT digits of 16 and 32 points at n = 2^24 (the paper's
    # radix sweep, Table 4, is at 2^24): passes of 2^8 = 16 x 16 (both digits
    # as tcgen05 products) against passes of 2^10 = 32 x 32 for 20 of the 24
    # stages; errors against the complex128 plan on two transforms
    n, batch = 1 << 24, 8
    gen = torch.Generator(device=dev).manual_seed(25)
    x = torch.randn(batch, n, dtype=torch.complex64, device=dev, generator=gen)
    y = torch.empty_like(x)
    with M.Plan(n, 2, M.FFT_C128, M.FFT_FORWARD) as pr:
        xr = x[:2].to(torch.complex128)
        yr = torch.empty_like(xr)
        pr.exec(xr, yr, stream)
    row = {"config": f"tensor-core radix sweep, c64 n=2^24 batch {batch} forward"}
    for form, fname in ((M.FFT_FORM_TC_FP16, "fp16"), (M.FFT_FORM_TC_BF16, "bf16")):
        for sched, key in (("8,8,8", "radix16"), ("10,10,4", "radix32")):
            p = M.Plan(n, batch, M.FFT_C64, M.FFT_FORWARD, form, sched)
            ms = _time(torch, stream, lambda: p.exec(x, y, stream), 3)
            M.fft_plan_check(p.handle)
            row[f"{fname}_{key}_ms"] = round(ms, 3)
            row[f"{fname}_{key}_rel_err"] = rel(y[:2], yr)
            p.close()
    p = M.Plan(n, batch, M.FFT_C64, M.FFT_FORWARD)
    row["fp32_default_ms"] = round(_time(torch, stream, lambda: p.exec(x, y, stream), 3), 3)
    p.close()
    _emit(row)
    del x, y, xr, yr

    # density-matrix gating by hyper-cube transpose: 14 qubits (2^28 elements,
    # larger than L2), in place; algorithmic bytes = one read + one write;
    # flops = the two 2^q x 2^q complex products per block
    nq = 14
    for f64 in (True, False):
        tdt = torch.complex128 if f64 else torch.complex64
        eb = 16 if f64 else 8
        gen = torch.Generator(device=dev).manual_seed(14)
        rho = torch.randn(1 << nq, 1 << nq, dtype=tdt, device=dev, generator=gen)
        for qubits in ([0], [13], [1, 12], [1, 6, 12]):
            q = len(qubits)
            u = np.linalg.qr(np.random.default_rng(q).standard_normal((1 << q, 1 << q)))[0].astype(np.complex128)
            ms = _time(torch, stream, lambda: M.dm_gate(rho, qubits, u, stream), 10)
            elems = float(1 << (2 * nq))
            gbs = 2 * elems * eb / (ms * 1e-3) / 1e9
            flops = elems / (1 << (2 * q)) * 2 * (1 << (3 * q)) * 8
            _emit({"config": f"density-matrix gate, {nq} qubits, qubits {qubits}, {'c128' if f64 else 'c64'}",
                   "ms": round(ms, 3), "gbs": round(gbs, 1),
                   frac_key: round(gbs / hbm, 4),
                   "gflops": round(flops / (ms * 1e-3) / 1e9, 1)})
        del rho


def max_over_ranks(value: float, dist, device) -> float:
    """The slowest rank's time (the job's time)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_case(args):
    """A small case for ncu captures of the complex64 kernels."""
    import torch
    import paper_0803_2386_gb300 as M
    torch.manual_seed(0)
    if args.case == "nd2d":  # 2-D complex64 4096 x 4096 x 2 (256 MiB): last axis, then two axis passes
        dims = (4096, 4096)
        gen = torch.Generator(device="cuda").manual_seed(2)
        x = torch.randn((2,) + dims, dtype=torch.complex64, device="cuda", generator=gen)
        y = torch.empty_like(x)
        with M.PlanND(dims, 2, M.FFT_C64, M.FFT_FORWARD) as p:
            for _ in range(args.steps):
                p.exec(x, y)
            torch.cuda.synchronize()
            M.fft_plan_check(p.handle)
        print("ok")
        return 0
    if args.case == "dm":  # density-matrix gate: 13 qubits, complex64 (512 MiB), qubit 0
        import numpy as np
        gen = torch.Generator(device="cuda").manual_seed(13)
        rho = torch.randn(1 << 13, 1 << 13, dtype=torch.complex64, device="cuda", generator=gen)
        u = np.linalg.qr(np.random.default_rng(0).standard_normal((2, 2)))[0].astype(np.complex128)
        for _ in range(3):
            M.dm_gate(rho, [0], u)
        torch.cuda.synchronize()
        print("ok")
        return 0
    form = {"c64": M.FFT_FORM_PLAIN, "tc_fp16": M.FFT_FORM_TC_FP16, "tc_bf16": M.FFT_FORM_TC_BF16,
            "tc32": M.FFT_FORM_TC_FP16, "c64_256": M.FFT_FORM_PLAIN,
            "c128": M.FFT_FORM_PLAIN, "df64": M.FFT_FORM_DF64, "c64_cluster": M.FFT_FORM_PLAIN,
            "c64_rows": M.FFT_FORM_PLAIN, "c1": M.FFT_FORM_PLAIN}[args.case]
    if args.case == "c1":  # one complex128 transform of 2^10 points (latency)
        n, batch = 1 << 10, 1
        x = torch.randn(batch, n, dtype=torch.complex128, device="cuda")
        y = torch.empty_like(x)
        p = M.Plan(n, batch, M.FFT_C128, M.FFT_FORWARD, form)
    elif args.case == "c64_rows":  # single-pass transforms (row tiles only)
        n, batch = 1 << 10, 1 << 16
        x = torch.randn(batch, n, dtype=torch.complex64, device="cuda")
        y = torch.empty_like(x)
        p = M.Plan(n, batch, M.FFT_C64, M.FFT_FORWARD, form)
    elif args.case == "c64_256":  # single-pass complex64 transforms of 256 points (warp-shuffle tiles), 256 MiB
        n, batch = 256, 1 << 17
        x = torch.randn(batch, n, dtype=torch.complex64, device="cuda")
        y = torch.empty_like(x)
        p = M.Plan(n, batch, M.FFT_C64, M.FFT_FORWARD, form)
    elif args.case == "tc32":  # complex64 n = 2^20 x 32 (256 MiB), two passes of 32 x 32 tensor-core digits
        n, batch = 1 << 20, 32
        x = torch.randn(batch, n, dtype=torch.complex64, device="cuda")
        y = torch.empty_like(x)
        p = M.Plan(n, batch, M.FFT_C64, M.FFT_FORWARD, form, "10,10;chunk=32")
    elif args.case in ("c128", "df64"):
        n, batch = 1 << 20, 16
        x = torch.randn(batch, n, dtype=torch.complex128, device="cuda")
        y = torch.empty_like(x)
        p = M.Plan(n, batch, M.FFT_C128, M.FFT_FORWARD, form)
    else:
        n, batch = 1 << 16, 512
        x = torch.randn(batch, n, dtype=torch.complex64, device="cuda")
        y = torch.empty_like(x)
        sched = "cluster" if args.case == "c64_cluster" else "8,8;chunk=512"
        p = M.Plan(n, batch, M.FFT_C64, M.FFT_FORWARD, form, sched)
        print(M.fft_plan_describe(p.handle))
    for _ in range(3):
        p.exec(x, y)
    M.fft_plan_check(p.handle)
    p.close()
    print("ok")
    return 0


def main():
    args = parse()
    if args.case:
        return run_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_moafft(args)


if __name__ == "__main__":
    sys.exit(main())
