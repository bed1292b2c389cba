#!/usr/bin/env python
"""MACH-HOOI benchmark on GB300.

One step = one whole decomposition of the workload: the Bernoulli coin over
the dense tensor (mach_sample: Philox sampler + per-mode orderings), HOSVD
initialisation, the HOOI sweeps and the core (mach_hooi).  Inputs are seeded
synthetic tensors resident in HBM before the timed region; the default
workload is the single large decomposition: 1000 x 1000 x 1000 FP32 (4 GB,
larger than the 129 MB L2, so no flush is needed), Tucker rank (10,10,10),
5% noise, p = 0.01, 20 sweeps, FP32 sweep arithmetic.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
instead (bounded sample, extrapolated; no GPU work).
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
sys.path.insert(0, ROOT)

METRIC = "Tucker decomps/sec + sampler HBM GB/s vs plain FP64 form at ≤1e-5 err; p50/p99"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mach", choices=["mach", "reference"])
    ap.add_argument("--workload", default="large_fp32", choices=["large_fp32", "plain_fp64"])
    ap.add_argument("--prec", default=None, help="fp32 | fp64 (default: the workload's)")
    ap.add_argument("--scale", type=int, default=1000, help="edge of the large workload (1000 = full size)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-slab", type=int, default=50, help="timeticks of the oracle's bounded sample")
    return ap.parse_args()


def workload(args):
    from paper_0909_4969_gb300 import synth
    if args.workload == "plain_fp64":
        w = synth.config_plain_fp64()
    else:
        w = synth.config_large_fp32(args.scale)
    prec = args.prec or w.precision
    return w, prec


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
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
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names[1:], parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def traffic_record(kernel: str):
    """dram bytes per launch from the committed ncu summary, if the kernel's
    source has not changed since it was captured (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)[kernel]
        src = os.path.join(ROOT, "paper_0909_4969_gb300", "csrc", rec["source"])
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if sha != rec["source_sha"]:
            return None
        return rec
    except Exception:
        return None


# ----------------------------------------------------------------------------
# oracle timing (cpu_baseline and --impl reference): spawned subprocess
# ----------------------------------------------------------------------------
ORACLE_SNIPPET = r"""
import os, sys, time, json
sys.path.insert(0, %(root)r)
from oracle import mach_oracle as O
from paper_0909_4969_gb300 import synth
spec = synth.TuckerSpec(%(dims)r, %(ranks)r, "gaussian", %(noise)r, %(seed)r, %(dtype)r)
X, _, _ = synth.tucker_numpy(spec)
O.build_oracle_lib()
t0 = time.perf_counter()
S, G, A = O.mach_hooi(X, spec.ranks, %(p)r, %(seed)r, %(sweeps)r)
t1 = time.perf_counter()
print(json.dumps({"seconds": t1 - t0, "kept": int(S.idx.size)}))
"""


def oracle_seconds(w, slab: int):
    """Time the oracle (single thread) end to end on the workload restricted to
    its first `slab` entries of the last mode; returns (seconds, sample text,
    scale factor to one full decomposition)."""
    dims = list(w.spec.dims)
    full_last = dims[-1]
    dims[-1] = min(slab, full_last)
    code = ORACLE_SNIPPET % dict(root=ROOT, dims=tuple(dims), ranks=tuple(w.spec.ranks), noise=w.spec.noise,
                                 seed=w.spec.seed, dtype=w.spec.dtype, p=w.p, sweeps=w.sweeps)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError("oracle subprocess failed: " + out.stderr[-2000:])
    res = json.loads(out.stdout.strip().splitlines()[-1])
    scale = full_last / dims[-1]
    sample = ("oracle end to end (coin, HOSVD init, %d sweeps, core) on the first %d of %d timeticks "
              "(%s, %d kept), time x %.1f" % (w.sweeps, dims[-1], full_last, "x".join(map(str, dims)),
                                              res["kept"], scale))
    return res["seconds"], sample, scale


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w, prec = workload(args)
    times = []
    sample = ""
    slab = max(1, min(args.cpu_slab, 20))
    for _ in range(args.warmup if args.warmup < 1 else 0):
        pass
    for _ in range(max(1, args.steps)):
        sec, sample, scale = oracle_seconds(w, slab)
        times.append(sec * scale)
    per = statistics.mean(times)
    value = 1.0 / per
    line = {"metric": METRIC, "value": value, "unit": "decompositions/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": len(times), "warmup": 0, "ms_per_step": per * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(w, "fp64"),
            "cpu_baseline": {"value": value, "unit": "decompositions/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "decompositions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def config_dict(w, prec):
    return {"workload": w.name, "dims": list(w.spec.dims), "ranks": list(w.spec.ranks), "p": w.p,
            "sweeps": w.sweeps, "noise": w.spec.noise, "core": w.spec.core, "input_dtype": w.spec.dtype,
            "prec": prec, "init": "HOSVD", "l2": "inputs larger than L2 (no flush)"
            if math.prod(w.spec.dims) * (4 if w.spec.dtype == "float32" else 8) > 129e6 else "L2 flushed"}


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__ as ge
    if rank == 0:
        ge.build()
    if world > 1:
        dist.barrier()
    ge.build()
    from paper_0909_4969_gb300 import mach, synth

    lib = mach.load()
    w, prec = workload(args)
    spec = w.spec
    # replicas: each rank decomposes its own tensor of the same workload
    spec_r = synth.TuckerSpec(spec.dims, spec.ranks, spec.core, spec.noise, spec.seed + rank, spec.dtype)
    X, _, _ = synth.tucker_torch(spec_r, device="cuda")
    torch.cuda.synchronize()
    ranks = spec.ranks
    N = X.numel()
    flush = None
    if N * X.element_size() <= 256 * 2 ** 20:
        flush = torch.empty(64 * 2 ** 20, dtype=torch.float32, device="cuda")   # 256 MB > L2

    last_stats = {}

    def step(x):
        s = mach.sample(x, w.p, spec_r.seed)
        G, A = s.hooi(ranks, w.sweeps, prec)
        last_stats.clear()
        last_stats.update(s.stats())
        s.free()
        return G, A

    for _ in range(max(0, args.warmup)):
        step(X)
        if flush is not None:
            flush.zero_()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    lib.mach_profile_enable(1)
    launches0 = lib.mach_launch_count()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    step_ms = []
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        G, A = step(X)
        b.record(stream)
        if flush is not None:
            flush.zero_()
        step_ms.append((a, b))
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    launches = lib.mach_launch_count() - launches0
    total_ms = e0.elapsed_time(e1)
    per_step = [a.elapsed_time(b) for a, b in step_ms]
    tmax = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    total_ms = float(tmax.item())
    value = world * args.steps / (total_ms / 1e3)

    # per-kernel-class profile (library-recorded CUDA events on this stream)
    prof = {}
    for kind, name in enumerate(["sampler", "ttm_chain", "leading_lsv", "mode_orderings", "hosvd_gram"]):
        ms = mach.ctypes.c_double()
        n = mach.ctypes.c_int64()
        by = mach.ctypes.c_double()
        lib.mach_profile_query(kind, mach.ctypes.byref(ms), mach.ctypes.byref(n), mach.ctypes.byref(by))
        prof[name] = {"ms": ms.value, "launches": n.value, "bytes": by.value}
    lib.mach_profile_enable(0)
    hbm_peak, peak_kind = measured_peaks()
    dom = max(("sampler", "ttm_chain"), key=lambda k: prof[k]["ms"])
    d = prof[dom]
    achieved = (d["bytes"] / max(d["launches"], 1)) / (d["ms"] / max(d["launches"], 1) / 1e3) / 1e9 if d["ms"] else 0
    samp = prof["sampler"]
    samp_gbs = (samp["bytes"] / max(samp["launches"], 1)) / (samp["ms"] / max(samp["launches"], 1) / 1e3) / 1e9 \
        if samp["ms"] else 0.0
    tr = traffic_record(dom)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "peak_source": peak_kind,
                "traffic": (tr["dram_bytes_per_unit"] * (d["bytes"] / max(d["launches"], 1)) if tr else None),
                "algorithmic_bytes_per_launch": d["bytes"] / max(d["launches"], 1),
                "avg_launch_ms": d["ms"] / max(d["launches"], 1)}

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        host = torch.empty(X.shape, dtype=X.dtype, pin_memory=True)
        host.copy_(X)
        xdev = torch.empty_like(X)
        h2d = host.numel() * host.element_size()
        d2h = 0
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.e2e_steps):
            xdev.copy_(host, non_blocking=True)
            G, A = step(xdev)
            outs = [G.cpu()] + [a.cpu() for a in A]
            d2h = sum(o.numel() * o.element_size() for o in outs)
        f1.record(stream)
        torch.cuda.synchronize()
        ems = f0.elapsed_time(f1)
        et = torch.tensor([ems], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(et, op=dist.ReduceOp.MAX)
        e2e = {"value": world * args.e2e_steps / (float(et.item()) / 1e3), "unit": "decompositions/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
        del host, xdev

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            sec, sample, scale = oracle_seconds(w, args.cpu_slab)
            cpu = {"value": 1.0 / (sec * scale), "unit": "decompositions/s", "cores": 1, "kind": "oracle",
                   "sample": sample}
        except Exception as ex:  # report, never fail the bench line
            cpu = {"value": None, "unit": "decompositions/s", "cores": 1, "kind": "oracle", "sample": str(ex)[:300]}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "decompositions/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "f64",
                "data": "synthetic", "config": config_dict(w, prec),
                "p50_ms": statistics.median(per_step),
                "p99_ms": sorted(per_step)[max(0, math.ceil(0.99 * len(per_step)) - 1)],
                "sampler_gbs": samp_gbs, "sampler_frac_of_hbm": samp_gbs / hbm_peak,
                "roofline": roofline, "profile_ms_per_step": {k: v["ms"] / args.steps for k, v in prof.items()},
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
                "eigensolver": last_stats}
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
