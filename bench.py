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

DTYPE_NAME = {"fp32": "f32", "fp64": "f64", "bf16_refine": "bf16+f32"}
METRIC = "Tucker decomps/sec + sampler HBM GB/s vs plain FP64 form at ≤1e-5 err; p50/p99"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mach", choices=["mach", "reference"])
    ap.add_argument("--workload", default="large_fp32", choices=["large_fp32", "plain_fp64", "mixed_4way", "served", "batched",
                                                       "tucker2_sensor"])
    ap.add_argument("--requests", type=int, default=400, help="served: requests in the timed run")
    ap.add_argument("--slots", type=int, default=8, help="served / batched: concurrent slots")
    ap.add_argument("--budget-gb", type=float, default=48.0, help="served / batched: HBM budget")
    ap.add_argument("--batch", type=int, default=512, help="batched: number of tensors")
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
    elif args.workload == "tucker2_sensor":
        w = synth.config_tucker2_sensor()
    elif args.workload == "mixed_4way":
        w = synth.config_mixed_4way(200 if args.scale == 1000 else args.scale)
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
# replicas: every rank decomposes its own tensor; the job's time is the
# slowest rank's, the job's throughput all ranks' decompositions over it
# ----------------------------------------------------------------------------
def max_over_ranks(ms: float, world: int, device) -> float:
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(steps_per_rank: int, world: int, max_ms: float) -> float:
    return world * steps_per_rank / (max_ms / 1e3)


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
if %(keep)r is None:
    S, G, A = O.mach_hooi(X, spec.ranks, %(p)r, %(seed)r, %(sweeps)r)
else:
    S, G, A = O.mach_tucker2(X, spec.ranks, %(keep)r, %(p)r, %(seed)r, %(sweeps)r)
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
    keep = 2 if w.name.startswith("tucker2") else None   # the Tucker2 workload keeps the time mode whole
    code = ORACLE_SNIPPET % dict(root=ROOT, dims=tuple(dims), ranks=tuple(w.spec.ranks), noise=w.spec.noise,
                                 seed=w.spec.seed, dtype=w.spec.dtype, p=w.p, sweeps=w.sweeps, keep=keep)
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


# ----------------------------------------------------------------------------
# served stream and batched windows (through mach_server_* / mach_submit / mach_poll)
# ----------------------------------------------------------------------------
def _drain(srv, tickets):
    errs = []
    pending = list(tickets)
    while pending:
        rest = []
        for t in pending:
            r = srv.poll(t)
            if r is None:
                rest.append(t)
            else:
                errs.append(r[2])
        pending = rest
        if pending:
            time.sleep(0.0005)
    return errs


def run_served(args):
    """64 streams of 200 x 16 x 512 FP32 windows rotating by 0.01 rad per
    window, Poisson arrivals at 2000 windows/s, 10% of the requests resized to
    1000 x 32 x 4096 (cold start); p = 0.1, ranks (4, 4, 8), 3 warm sweeps.
    Windows come from a pre-generated device pool (4 per stream, 2 resized)."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_0909_4969_gb300 import mach, synth
    mach.load()
    n_streams, pool_w = 64, 4
    small, big = (200, 16, 512), (1000, 32, 4096)
    ranks, p, sweeps = (4, 4, 8), 0.1, 3
    prec = args.prec or "fp32"
    gens = [synth.StreamStateTorch(s, small, ranks, seed=1) for s in range(n_streams)]
    pool = [[g.next_window(0.01, 0.05) for _ in range(pool_w)] for g in gens]
    bigs = [synth.tucker_torch(synth.TuckerSpec(big, ranks, "gaussian", 0.05, 100 + k, "float32"))[0]
            for k in range(2)]
    torch.cuda.synchronize()

    def one_run(n, seed):
        sched = synth.served_schedule(n, n_streams, 2000.0, 0.10, seed, small, big)
        srv = mach.Server(int(args.budget_gb * 2 ** 30), args.slots)
        tickets = []
        t0 = time.perf_counter()
        for req in sched:
            delay = t0 + req.arrival_s - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            x = bigs[req.window % 2] if req.resized else pool[req.stream][req.window % pool_w]
            tickets.append(srv.submit(req.stream, x, ranks, p, req.seed, sweeps, prec))
        errs = _drain(srv, tickets)
        t1 = time.perf_counter()
        st = srv.stats()
        srv.close()
        return n / (t1 - t0), st, errs, t1 - t0, sum(r.resized for r in sched)

    one_run(max(32, 16 * args.warmup), 12345)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    value, st, errs, wall, n_big = one_run(args.requests, 7)
    clk = clocks.stop()
    line = {"metric": METRIC, "value": value, "unit": "decompositions/s", "n_gpus": 1, "steps": args.requests,
            "warmup": max(32, 16 * args.warmup), "ms_per_step": 1e3 / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAME.get(prec, prec),
            "data": "synthetic",
            "config": {"workload": "served_stream_64x200x16x512", "streams": n_streams, "window": list(small),
                       "resized_window": list(big), "resize_frac": 0.10, "rate_hz": 2000.0, "p": p,
                       "ranks": list(ranks), "sweeps": sweeps, "warm_start": True, "slots": args.slots,
                       "budget_gb": args.budget_gb, "requests": args.requests, "resized_requests": n_big,
                       "prec": prec},
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_in_flight": st["max_in_flight"],
            "wall_s": wall, "rel_err_median": statistics.median(errs), "rel_err_max": max(errs),
            "clocks": clk}
    print(json.dumps(line))
    return 0


def run_batched(args):
    """512 independent FP32 tensors of uneven sizes (hosts U{50..400}, types
    U{8..32}, timeticks log-uniform 64..2048), rank (4, 4, 8), 10% noise,
    p = 0.1, 10 sweeps.  The value is the one-launch form (every tensor
    sampled, then mach_hooi_batched); beside it the served form (all
    submitted at once to the server: continuous batching over `slots`
    streams) and the plain FP64 form (one decomposition at a time, FP64
    sweeps) on the same tensors."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_0909_4969_gb300 import mach, synth
    mach.load()
    ws = synth.config_batched(args.batch)
    xs = [synth.tucker_torch(w.spec)[0] for w in ws]
    torch.cuda.synchronize()
    ranks = (4, 4, 8)
    prec = args.prec or "fp32"

    def run(pr, slots, items):
        srv = mach.Server(int(args.budget_gb * 2 ** 30), slots)
        t0 = time.perf_counter()
        tickets = [srv.submit(b, x, ranks, 0.1, b, 10, pr) for b, x in items]
        errs = _drain(srv, tickets)
        t1 = time.perf_counter()
        st = srv.stats()
        srv.close()
        return len(items) / (t1 - t0), st, errs

    import concurrent.futures as cf
    sample_streams = [torch.cuda.Stream() for _ in range(args.slots)]

    def sample_slot(j, items):
        st = sample_streams[j]
        return [(b, mach.sample(x, 0.1, b, stream=st)) for b, x in items[j::len(sample_streams)]]

    def one_launch(items):
        # mach_sample per tensor (host threads on `slots` streams: each call
        # synchronises its own stream to size the kept set), then HOSVD start
        # + 10 sweeps + core of all of them in one persistent launch
        # (mach_hooi_batched)
        t0 = time.perf_counter()
        with cf.ThreadPoolExecutor(len(sample_streams)) as ex:
            parts = list(ex.map(lambda j: sample_slot(j, items), range(len(sample_streams))))
        samples = [smp for _, smp in sorted((t for part in parts for t in part), key=lambda t: t[0])]
        torch.cuda.synchronize()
        cores, facs = mach.hooi_batched(samples, ranks, 10)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        errs = [mach.error(x, cores[i], facs[i])[0] for i, (_, x) in enumerate(items)]
        flags = max(s.stats()["flags"] for s in samples)
        for s in samples:
            s.free()
        return len(items) / (t1 - t0), errs, flags

    items = list(enumerate(xs))
    one_launch(items[:32])
    run(prec, args.slots, items[:32])
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    value, errs, flags = one_launch(items)
    srv_value, st, srv_errs = run(prec, args.slots, items)
    clk = clocks.stop()
    plain, st64, errs64 = run("fp64", 1, items)
    line = {"metric": METRIC, "value": value, "unit": "decompositions/s", "n_gpus": 1, "steps": len(items),
            "warmup": 32, "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched_%d_uneven" % len(items), "ranks": list(ranks), "p": 0.1, "sweeps": 10,
                       "noise": 0.10, "form": "mach_sample per tensor (%d threads / streams) + mach_hooi_batched "
                       "(one launch)" % args.slots,
                       "total_input_gb": sum(x.numel() * 4 for x in xs) / 1e9},
            "rel_err_median": statistics.median(errs), "rel_err_max": max(errs), "device_flags": flags,
            "served_form": {"value": srv_value, "unit": "decompositions/s", "slots": args.slots,
                            "budget_gb": args.budget_gb, "prec": prec, "p50_ms": st["p50_ms"],
                            "p99_ms": st["p99_ms"], "max_in_flight": st["max_in_flight"],
                            "rel_err_median": statistics.median(srv_errs), "rel_err_max": max(srv_errs)},
            "plain_fp64": {"value": plain, "unit": "decompositions/s", "slots": 1,
                           "rel_err_median": statistics.median(errs64), "rel_err_max": max(errs64)},
            "clocks": clk}
    print(json.dumps(line))
    return 0


def config_dict(w, prec):
    c = {"workload": w.name, "dims": list(w.spec.dims), "ranks": list(w.spec.ranks), "p": w.p,
         "sweeps": w.sweeps, "noise": w.spec.noise, "core": w.spec.core, "input_dtype": w.spec.dtype,
         "prec": prec, "init": "HOSVD", "l2": "inputs larger than L2 (no flush)"
         if math.prod(w.spec.dims) * (4 if w.spec.dtype == "float32" else 8) > 129e6 else "L2 flushed"}
    if w.name.startswith("tucker2"):
        c["decomposition"] = "Tucker2: ranks (%d, %d), mode 3 (time) kept whole; generator rank %s" % (
            w.spec.ranks[0], w.spec.ranks[1], list(w.spec.ranks))
    return c


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "served":
        return run_served(args)
    if args.workload == "batched":
        return run_batched(args)
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
    # decompositions run on a stream of their own (the library replays the
    # repeated HOOI sweeps as a captured CUDA graph, which the legacy default
    # stream does not allow)
    torch.cuda.set_stream(torch.cuda.Stream())
    ranks = spec.ranks
    N = X.numel()
    flush = None
    if N * X.element_size() <= 256 * 2 ** 20:
        flush = torch.empty(64 * 2 ** 20, dtype=torch.float32, device="cuda")   # 256 MB > L2

    last_stats = {}

    def step(x):
        s = mach.sample(x, w.p, spec_r.seed)
        if args.workload == "tucker2_sensor":
            G, A = s.tucker2((ranks[0], ranks[1], 0), 2, w.sweeps, prec)   # time mode kept whole
        else:
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
    total_ms = max_over_ranks(total_ms, world, "cuda")
    value = replica_throughput(args.steps, world, total_ms)

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

    # the sector-skipping sampler on the same resident input (outside the timed
    # region): its time, and the share of X's 32-byte sectors it has to read
    skip = None
    if w.spec.dtype in ("float32", "float64"):
        lib.mach_profile_enable(1)
        for _ in range(3):
            s2 = mach.sample(X, w.p, spec_r.seed, skip=True)
            s2.free()
        ms2 = mach.ctypes.c_double()
        n2 = mach.ctypes.c_int64()
        by2 = mach.ctypes.c_double()
        lib.mach_profile_query(0, mach.ctypes.byref(ms2), mach.ctypes.byref(n2), mach.ctypes.byref(by2))
        lib.mach_profile_enable(0)
        per = 4 if w.spec.dtype == "float32" else 8
        skip = {"ms": ms2.value / max(n2.value, 1), "sector_fraction_read": 1.0 - (1.0 - w.p) ** (32 // per),
                "vs_dense": samp["ms"] / max(samp["launches"], 1) / (ms2.value / max(n2.value, 1))
                if ms2.value else None}

    # end to end through the public API with host buffers
    e2e = None
    host_stream = None
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
            outs = [G.cpu()] + [a.cpu() for a in A if a is not None]
            d2h = sum(o.numel() * o.element_size() for o in outs)
        f1.record(stream)
        torch.cuda.synchronize()
        ems = f0.elapsed_time(f1)
        ems = max_over_ranks(ems, world, "cuda")
        e2e = {"value": replica_throughput(args.e2e_steps, world, ems), "unit": "decompositions/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
        # the sampler streaming X from host memory (mach_sample_host, 1 GiB
        # chunks overlapping the coin): the form for tensors larger than HBM
        del xdev
        hs = []
        for _ in range(2):
            h0 = torch.cuda.Event(enable_timing=True)
            h1 = torch.cuda.Event(enable_timing=True)
            h0.record(stream)
            sh = mach.sample(host, w.p, spec_r.seed)
            h1.record(stream)
            torch.cuda.synchronize()
            hs.append(h0.elapsed_time(h1))
            sh.free()
        host_stream = {"ms": min(hs), "input_gb_per_s": h2d / (min(hs) / 1e3) / 1e9,
                       "note": "mach_sample_host: coin + orderings of X held in pinned host memory"}
        del host

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
                "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAME.get(prec, prec),
                "data": "synthetic", "config": config_dict(w, prec),
                "p50_ms": statistics.median(per_step),
                "p99_ms": sorted(per_step)[max(0, math.ceil(0.99 * len(per_step)) - 1)],
                "sampler_gbs": samp_gbs, "sampler_frac_of_hbm": samp_gbs / hbm_peak, "sampler_skip": skip,
                "sampler_host_stream": host_stream,
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
