#!/usr/bin/env python
"""Benchmark: C-A CUR solves per second on GB300.

One step = one full C-A solve through the library's C ABI (all sweeps,
nucleus, Appendix F sampled error estimate) on a synthetic workload whose
inputs are already resident in HBM.  Default workload: the generated Cauchy
matrix a_ij = 1/(x_i - y_j), x ~ U[0,1], y ~ U[2,3], m = n = 65536 (never
materialised), k = 16, l = 24, 4 sweeps, error estimated on a 1000 x 1000
sample.  The strips and inputs fit in L2, so L2 is flushed (a 256 MiB write)
before every timed step and each step is timed with its own CUDA events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs independent replicas (one solve stream per GPU, no collective on
the data path); the reference arm runs the FP64 CPU oracle.
"""
from __future__ import annotations

import argparse
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

METRIC = "C-A CUR solves/s and gather GB/s vs plain GPU C-A at equal error; p50/p99 latency"
UNIT = "solves/s"

WORKLOADS = {
    "cauchy65536": dict(kind="cauchy", m=65536, n=65536, k=16, l=24, sweeps=4, q=1000, s=1000,
                        seed_off=2),
    "dense256": dict(kind="dense64", m=256, n=256, k=8, l=8, sweeps=3, q=256, s=256, seed_off=1),
    # stored FP32 32768^2 = G1 G2^T / 8 + N(0, 1e-4^2), full residual on the tensor cores
    "dense32768": dict(kind="dense32", m=32768, n=32768, k=64, l=96, sweeps=4, q=1000, s=1000,
                       seed_off=3, full=True),
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# FP64 FMA issue rate of a GB300 SM: 1.25 TFLOP/s nominal at the 2070 MHz
# maximum SM clock over 152 SMs is 2 FP64 FMA per SM per clock.
FP64_FMA_PER_SM_CLK = 2
SMS = 152


def fp64_peak_tflops(sm_mhz):
    return SMS * FP64_FMA_PER_SM_CLK * 2 * sm_mhz * 1e6 / 1e12


# ---------------------------------------------------------------------------
# inputs
# ---------------------------------------------------------------------------

def make_inputs(wl, rank=0):
    import workloads as W
    seed = W.BASE_SEED + wl["seed_off"] + 1000 * rank
    m, n, l = wl["m"], wl["n"], wl["l"]
    inp = {"J0": W.draw_indices(seed + 100, n, l),
           "rows": W.draw_indices(seed + 200, m, wl["q"], sort=True),
           "cols": W.draw_indices(seed + 300, n, wl["s"], sort=True)}
    if wl["kind"] == "cauchy":
        inp["x"], inp["y"] = W.cauchy_points(seed, m, n)
    else:
        inp["a"] = (W.factor_gaussian(seed, m, n, 64, 1e-4) if wl["kind"] == "dense32"
                    else W.lowrank_svd(seed, m, n, r=8, noise_std=1e-4))
    return inp


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
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
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, one thread, bounded sample
# ---------------------------------------------------------------------------

CPU_SNIPPET = r"""
import os, sys, time, json
sys.path.insert(0, {root!r})
import numpy as np
import oracle as O, workloads as W
sys.path.insert(0, {root!r})
from bench import WORKLOADS, make_inputs
wl = WORKLOADS[{wl!r}]
inp = make_inputs(wl, 0)
if wl["kind"] == "cauchy":
    src = O.Cauchy(inp["x"], inp["y"], "fp64")
else:
    src = O.Dense(inp["a"])
t0 = time.perf_counter(); n = 0; times = []
while True:
    t1 = time.perf_counter()
    O.cross_approximation(src, inp["J0"], k=wl["k"], sweeps=wl["sweeps"],
                          sample_rows=inp["rows"], sample_cols=inp["cols"], keep_trace=False)
    times.append(time.perf_counter() - t1); n += 1
    if (time.perf_counter() - t0 > {budget} and n >= {min_n}) or n >= {max_n}:
        break
print(json.dumps({{"n": n, "total_s": sum(times), "times": times}}))
"""


def run_oracle(wl_name, budget_s=12.0, min_n=1, max_n=1000):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = CPU_SNIPPET.format(root=ROOT, wl=wl_name, budget=budget_s, min_n=min_n, max_n=max_n)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=900)
    if r.returncode != 0:
        raise RuntimeError(f"oracle baseline failed: {r.stderr[-2000:]}")
    return json.loads(r.stdout.strip().splitlines()[-1])


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

def run_ours(args, wl_name):
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

    import paper_1611_01391_gb300 as L

    wl = WORKLOADS[wl_name]
    inp = make_inputs(wl, rank)
    m, n, k, l, sweeps = wl["m"], wl["n"], wl["k"], wl["l"], wl["sweeps"]
    stream = torch.cuda.Stream(dev)        # the library and torch share this stream
    torch.cuda.set_stream(stream)
    ctx = L.Context(local, stream=stream.cuda_stream)

    if wl["kind"] == "cauchy":
        xd = torch.from_numpy(inp["x"]).to(dev)
        yd = torch.from_numpy(inp["y"]).to(dev)
        src = L.make_source("cauchy", x=xd, y=yd)
    else:
        ad = torch.from_numpy(inp["a"]).to(dev)
        src = L.make_source("dense", a=ad)
    params, keep = L.make_params(k, l, sweeps, inp["J0"], resid_rows=inp["rows"],
                                 resid_cols=inp["cols"], profile=True,
                                 full_residual=wl.get("full", False))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def one_step():
        job = ctx.submit(src, params)
        return job

    # warm-up
    for _ in range(args.warmup):
        res = ctx.fetch(one_step(), l)
        assert res.info.status == 0, L.lra_status_str(res.info.status)

    clocks = ClockSampler(local)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clocks.start()
    time.sleep(0.3)
    evs = []
    infos = []
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        job = one_step()
        b.record(stream)
        evs.append((a, b))
        res = ctx.fetch(job, l)
        infos.append(res.info)
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter() - t_wall0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    for inf in infos:
        if inf.status != 0:
            raise RuntimeError(f"solve failed: {L.lra_status_str(inf.status)}")
    value = world * args.steps / (total_ms / 1e3)

    # ---- roofline of the dominant kernel class, from the live per-launch events
    t_mv = sum(i.t_maxvol_ms for i in infos)
    fl_mv = sum(i.maxvol_flops for i in infos)
    t_g = sum(i.t_gather_ms for i in infos)
    t_x = sum(i.t_cross_ms for i in infos)
    t_r = sum(i.t_resid_ms for i in infos)
    sm_mhz = clk.get("sm_mhz") or 2070.0
    peaks, peak_kind = _peaks()
    fp64_peak = fp64_peak_tflops(sm_mhz)
    achieved = fl_mv / (t_mv / 1e3) / 1e12 if t_mv > 0 else 0.0
    # gathers: bytes written (strips) per solve; generated entries read nothing
    strips_bytes = ((sweeps + 1) * m * l + sweeps * l * n) * 4
    gather_gbs = strips_bytes * len(infos) / (t_g / 1e3) / 1e9 if t_g > 0 else 0.0

    # ---- end to end through the public API from host buffers
    e2e = None
    if wl["kind"] == "cauchy":
        xh = torch.from_numpy(inp["x"]).pin_memory()
        yh = torch.from_numpy(inp["y"]).pin_memory()
        xd2 = torch.empty_like(xd)
        yd2 = torch.empty_like(yd)
        src2 = L.make_source("cauchy", x=xd2, y=yd2)
        h2d = xh.numel() * 4 + yh.numel() * 4 + 4 * (l + wl["q"] + wl["s"])
        d2h = 4 * 2 * l + 8 * l * l + 8 * l + 144
        ts = []
        for it in range(args.warmup + args.steps):
            flush.zero_()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            xd2.copy_(xh, non_blocking=True)
            yd2.copy_(yh, non_blocking=True)
            r2 = ctx.fetch(ctx.submit(src2, params), l)
            assert r2.info.status == 0
            t1 = time.perf_counter()
            if it >= args.warmup:
                ts.append(t1 - t0)
        e2e = {"value": len(ts) / sum(ts) * world, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}
    else:
        ah = torch.from_numpy(inp["a"]).pin_memory()
        ad2 = torch.empty_like(ad)
        src2 = L.make_source("dense", a=ad2)
        h2d = ah.numel() * ah.element_size() + 4 * (l + wl["q"] + wl["s"])
        d2h = 4 * 2 * l + 8 * l * l + 8 * l + 144
        ts = []
        for it in range(min(args.warmup, 1) + args.steps):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            ad2.copy_(ah, non_blocking=True)
            r2 = ctx.fetch(ctx.submit(src2, params), l)
            assert r2.info.status == 0
            t1 = time.perf_counter()
            if it >= min(args.warmup, 1):
                ts.append(t1 - t0)
        e2e = {"value": len(ts) / sum(ts) * world, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    lat = sorted(step_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl_name, "generator": wl["kind"], "m": m, "n": n, "k": k, "l": l,
                   "sweeps": sweeps, "error_sample": f"{wl['q']}x{wl['s']}",
                   "precision": "FP32 entries/strips, FP64 maxvol and cross, compensated FP32 residual products",
                   "l2": "flushed before every step (256 MiB write); steps timed individually",
                   "parallelism": f"replicas{world}"},
        "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)],
        "wall_s": t_wall,
        "gather_gbs": gather_gbs,
        "kernel_ms_per_step": {"maxvol": t_mv / len(infos), "gather": t_g / len(infos),
                               "inverse": sum(i.t_inverse_ms for i in infos) / len(infos),
                               "nucleus": t_x / len(infos), "resid": t_r / len(infos)},
        "roofline": {"kernel": "maxvol_kernel", "bound": "alu", "achieved": achieved,
                     "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak if fp64_peak else None,
                     "traffic": captured_traffic("k_maxvol.cu", f"maxvol_{wl_name}.md"),
                     "traffic_note": "DRAM bytes per maxvol launch from the committed ncu capture (null if the kernel changed since)",
                     "peak_source": f"FP64 FMA rate: {SMS} SMs x {FP64_FMA_PER_SM_CLK} FMA/clk x median SM clock {sm_mhz:.0f} MHz"},
        "gpu_launches": int(sum(i.kernel_launches for i in infos)),
        "clocks": clk,
        "e2e": e2e,
        "swaps_per_solve": statistics.mean(i.swaps_total for i in infos),
        "full_rel_err": infos[-1].full_rel_err,
        "est_rel_err": infos[-1].est_rel_err,
    }
    if wl.get("full"):
        t_fr = sum(i.t_fullres_ms for i in infos) / len(infos)
        gbs = m * n * 4 / (t_fr / 1e3) / 1e9 if t_fr > 0 else 0.0
        line["kernel_ms_per_step"]["full_residual"] = t_fr
        line["roofline_full_residual"] = {
            "kernel": "fullres_kernel (+ operand split kernels)", "bound": "hbm", "achieved": gbs,
            "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
            "traffic": captured_traffic("k_fullres.cu", f"fullres_{wl_name}.md"),
            "peak_source": f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
            "algorithmic_bytes": m * n * 4}
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        if world == 1:
            try:
                ob = run_oracle(wl_name)
                line["cpu_baseline"] = {"value": ob["n"] / ob["total_s"], "unit": UNIT, "cores": 1,
                                        "kind": "oracle",
                                        "sample": f"{ob['n']} full solve(s) of the same workload, FP64 numpy, 1 thread"}
            except Exception as e:  # report, do not hide
                line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                        "sample": f"failed: {e}"}
        print(json.dumps(line), flush=True)


def run_profile_solves(args, wl_name):
    """N solves of the workload and nothing else: the command that ncu
    captures (launch list, per-kernel counters)."""
    import torch
    import paper_1611_01391_gb300 as L
    wl = WORKLOADS[wl_name]
    inp = make_inputs(wl, 0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = L.Context(0, stream=stream.cuda_stream)
    if wl["kind"] == "cauchy":
        xd = torch.from_numpy(inp["x"]).cuda()
        yd = torch.from_numpy(inp["y"]).cuda()
        src = L.make_source("cauchy", x=xd, y=yd)
    else:
        ad = torch.from_numpy(inp["a"]).cuda()
        src = L.make_source("dense", a=ad)
    params, keep = L.make_params(wl["k"], wl["l"], wl["sweeps"], inp["J0"], resid_rows=inp["rows"],
                                 resid_cols=inp["cols"], full_residual=wl.get("full", False))
    for _ in range(args.profile_solves):
        res = ctx.fetch(ctx.submit(src, params), wl["l"])
        if res.info.status != 0:
            raise RuntimeError(L.lra_status_str(res.info.status))
    ctx.close()
    print(f"profile solves done: {args.profile_solves} x {wl_name}", flush=True)


def captured_traffic(kernel_file, summary):
    """DRAM bytes per launch from a committed ncu summary, or None when the
    kernel source changed since that capture (its sha256 is recorded)."""
    import hashlib
    try:
        text = open(os.path.join(ROOT, "profiles", summary)).read()
        src = open(os.path.join(ROOT, "paper_1611_01391_gb300", "csrc", kernel_file), "rb").read()
    except OSError:
        return None
    fields = dict(ln.split(":", 1) for ln in text.splitlines() if ln.startswith(("traffic_bytes_per_launch:", "source_sha256:")))
    if fields.get("source_sha256", "").strip() != hashlib.sha256(src).hexdigest():
        return None
    return float(fields["traffic_bytes_per_launch"])


def run_reference(args, wl_name):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = WORKLOADS[wl_name]
    total = args.warmup + args.steps
    ob = run_oracle(wl_name, budget_s=1e9, min_n=total, max_n=total)
    times = ob["times"][args.warmup:]
    value = len(times) / sum(times)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": wl_name, "generator": wl["kind"], "m": wl["m"], "n": wl["n"],
                       "k": wl["k"], "l": wl["l"], "sweeps": wl["sweeps"],
                       "error_sample": f"{wl['q']}x{wl['s']}"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{len(times)} full solve(s) per timed run, FP64 numpy, 1 thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="cauchy65536")
    ap.add_argument("--profile-solves", type=int, default=0,
                    help="run this many solves and exit (the command ncu captures)")
    args = ap.parse_args()
    if args.profile_solves:
        run_profile_solves(args, args.workload)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args, args.workload)
    else:
        run_ours(args, args.workload)


if __name__ == "__main__":
    main()
