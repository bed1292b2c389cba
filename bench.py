#!/usr/bin/env python
"""MACH-HOOI benchmark on GB300.

One step = one whole decomposition of the workload: the Bernoulli coin over
the dense tensor (mach_sample: Philox sampler + per-mode orderings), HOSVD
initialisation, the HOOI sweeps and the core (mach_hooi).  Inputs are seeded
synthetic tensors resident in HBM before the timed region; the default
workload is the single large decomposition: 1000 x 1000 x 1000 FP32 (4 GB,
larger than the 129 MB L2, so no flush is needed), Tucker rank (10,10,10),
5% noise, p = 0.01, 20 sweeps, FP32 sweep arithmetic.

Besides the timed FP32 form, the default line carries:
  plain_fp64   the same decomposition with FP64 sweep arithmetic (the plain
               FP64 GPU form), timed the same way;
  accuracy     FP32 against FP64 and both against the FP64 CPU oracle run
               once at full size on the same input (subspace distance per
               mode, sign-fixed core, reconstruction error of Section 4);
  cpu_baseline that full-size oracle run (its time, one host core);
  batched      512 uneven windows in one persistent launch, beside the plain
               FP64 form on a subset and checked against the oracle;
  served       the served tensor stream (continuous batching), p50 / p99.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
instead: every step is one whole decomposition of the workload at full size,
the steps running as concurrent processes on the host cores (no GPU work).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DTYPE_NAME = {"fp32": "f32", "fp64": "f64", "bf16_refine": "bf16+f32"}
METRIC = "Tucker decomps/sec + sampler HBM GB/s vs plain FP64 form at ≤1e-5 err; p50/p99"
FALLBACK_HBM_GBS = 6800.0
PROF_KINDS = ["sampler", "ttm_chain", "leading_lsv", "mode_orderings", "hosvd_gram"]


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
    ap.add_argument("--fp64-steps", type=int, default=2, help="timed steps of the plain FP64 form")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the full-size oracle run")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 form")
    ap.add_argument("--no-sub", action="store_true", help="skip the batched and served sub-results")
    ap.add_argument("--cpu-slab", type=int, default=50,
                    help="mixed_4way only: last-mode slab the oracle decomposes (the full 4-way tensor is too "
                         "large for it)")
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


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def scratch_dir() -> str:
    base = "/dev/shm" if os.path.isdir("/dev/shm") and os.access("/dev/shm", os.W_OK) else None
    return tempfile.mkdtemp(prefix="mach_bench_", dir=base)


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
# comparison metrics (reporting only; the decompositions come from libmach
# and from the oracle)
# ----------------------------------------------------------------------------
def _np(a):
    import numpy as np
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.asarray(a, dtype=np.float64)


def subspace_distance(A, B) -> float:
    """||A A^T - B B^T||_F / sqrt(2 r) for orthonormal I x r A, B, formed as
    ||B - A (A^T B)||_F / sqrt(r) (the same quantity for orthonormal bases,
    without the I x I matrices and without cancellation)."""
    import numpy as np
    A, B = _np(A), _np(B)
    return float(np.linalg.norm(B - A @ (A.T @ B)) / math.sqrt(A.shape[1]))


def sign_fixed_core(G, factors):
    import numpy as np
    G = _np(G).copy()
    for k, A in enumerate(factors):
        A = _np(A)
        s = np.ones(A.shape[1])
        for j in range(A.shape[1]):
            i = int(np.argmax(np.abs(A[:, j])))
            s[j] = -1.0 if A[i, j] < 0 else 1.0
        shape = [1] * G.ndim
        shape[k] = -1
        G = G * s.reshape(shape)
    return G


def compare(Ga, Aa, Gb, Ab) -> dict:
    import numpy as np
    dist = [subspace_distance(a, b) for a, b in zip(Aa, Ab)]
    ca, cb = sign_fixed_core(Ga, Aa), sign_fixed_core(Gb, Ab)
    return {"subspace_distance_max": max(dist), "subspace_distance": dist,
            "core_rel_diff": float(np.linalg.norm(ca - cb) / np.linalg.norm(cb))}


# ----------------------------------------------------------------------------
# the oracle (cpu_baseline and --impl reference): spawned subprocesses
# ----------------------------------------------------------------------------
ORACLE_SNIPPET = r"""
import os, sys, time, json
sys.path.insert(0, %(root)r)
import numpy as np
from oracle import mach_oracle as O
X = np.load(%(xpath)r, mmap_mode="r")
if %(slab)r:
    X = np.ascontiguousarray(X[..., :%(slab)r])
O.build_oracle_lib()
t0 = time.perf_counter()
if %(keep)r is None:
    S, G, A = O.mach_hooi(X, %(ranks)r, %(p)r, %(seed)r, %(sweeps)r)
else:
    S, G, A = O.mach_tucker2(X, %(ranks)r, %(keep)r, %(p)r, %(seed)r, %(sweeps)r)
t1 = time.perf_counter()
if %(out)r:
    np.savez(%(out)r, G=G, **{"A%%d" %% k: a for k, a in enumerate(A)})
print(json.dumps({"seconds": t1 - t0, "kept": int(S.idx.size)}))
"""


def oracle_proc(xpath, w, out=None, slab=0, threads=1):
    keep = 2 if w.name.startswith("tucker2") else None   # the Tucker2 workload keeps the time mode whole
    code = ORACLE_SNIPPET % dict(root=ROOT, xpath=xpath, slab=int(slab), ranks=tuple(w.spec.ranks),
                                 p=w.p, seed=w.spec.seed, sweeps=w.sweeps, keep=keep, out=out)
    env = dict(os.environ, OMP_NUM_THREADS=str(threads), OPENBLAS_NUM_THREADS=str(threads),
               MKL_NUM_THREADS=str(threads))
    return subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                            text=True, env=env)


def oracle_result(proc, timeout=3600):
    out, err = proc.communicate(timeout=timeout)
    if proc.returncode != 0:
        raise RuntimeError("oracle subprocess failed: " + err[-2000:])
    return json.loads(out.strip().splitlines()[-1])


def load_oracle_decomp(path, d):
    import numpy as np
    z = np.load(path)
    return z["G"], [z["A%d" % k] for k in range(d)]


def run_reference(args):
    """Every step is one whole decomposition of the workload by the oracle at
    full size (the mixed 4-way tensor: a last-mode slab, stated), on the
    host's cores: the K steps run as concurrent single-threaded processes.
    The value is K over the wall time from the first start to the last end."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np
    import torch
    from paper_0909_4969_gb300 import synth
    w, _ = workload(args)
    cores = host_cores()
    torch.set_num_threads(cores)
    X, _, _ = synth.tucker_torch(w.spec, device="cpu")
    tmp = scratch_dir()
    try:
        xpath = os.path.join(tmp, "x.npy")
        np.save(xpath, X.numpy())
        del X
        slab = args.cpu_slab if w.name.startswith("mixed_4way") else 0
        K = max(1, args.steps)
        par = max(1, min(K, 2 * cores))
        # warm-up: the oracle's coin library is built and the input paged in
        from oracle import mach_oracle as O
        O.build_oracle_lib()
        secs = []
        kept = 0
        t0 = time.perf_counter()
        pending = list(range(K))
        running = []
        while pending or running:
            while pending and len(running) < par:
                pending.pop()
                running.append(oracle_proc(xpath, w, slab=slab))
            res = oracle_result(running.pop(0))
            secs.append(res["seconds"])
            kept = res["kept"]
        wall = time.perf_counter() - t0
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    value = K / wall
    dims = list(w.spec.dims)
    if slab:
        dims[-1] = min(slab, dims[-1])
    sample = ("%d whole oracle decompositions (coin, HOSVD init, %d sweeps, core) of %s (%d kept), %d at a time as "
              "single-threaded processes on %d host cores; mean %.1f s each" %
              (K, w.sweeps, "x".join(map(str, dims)) + (" (slab of the %s tensor)" % "x".join(map(str, w.spec.dims))
                                                      if slab else " (full size)"),
               kept, par, cores, statistics.mean(secs)))
    line = {"metric": METRIC, "value": value, "unit": "decompositions/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": K, "warmup": args.warmup, "ms_per_step": wall * 1e3 / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(w, "fp64"),
            "cpu_baseline": {"value": value, "unit": "decompositions/s", "cores": min(par, cores), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "decompositions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "note": "warm-up = building the oracle's coin library and paging the input in (a CPU program has no "
                    "device warm-up)"}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------
# served stream and batched windows (through mach_server_* / mach_submit / mach_poll)
# ----------------------------------------------------------------------------
def _drain(srv, tickets):
    out = {}
    pending = list(tickets)
    while pending:
        rest = []
        for t in pending:
            r = srv.poll(t)
            if r is None:
                rest.append(t)
            else:
                out[t] = r
        pending = rest
        if pending:
            time.sleep(0.0005)
    return [out[t] for t in tickets]


def served_results(args, requests=None):
    """64 streams of 200 x 16 x 512 FP32 windows rotating by 0.01 rad per
    window, Poisson arrivals at 2000 windows/s, 10% of the requests resized to
    1000 x 32 x 4096 (cold start); p = 0.1, ranks (4, 4, 8), 3 warm sweeps.
    Windows come from a pre-generated device pool (4 per stream, 2 resized).
    One resized window decomposed by the server is checked against the
    oracle (cold HOSVD start + 3 sweeps)."""
    import torch
    from paper_0909_4969_gb300 import mach, synth
    requests = requests or args.requests
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
        res = _drain(srv, tickets)
        t1 = time.perf_counter()
        st = srv.stats()
        srv.close()
        return n / (t1 - t0), st, [r[2] for r in res], t1 - t0, sum(r.resized for r in sched)

    one_run(max(32, 16 * args.warmup), 12345)
    value, st, errs, wall, n_big = one_run(requests, 7)
    out = {"value": value, "unit": "decompositions/s", "requests": requests, "resized_requests": n_big,
           "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_in_flight": st["max_in_flight"], "wall_s": wall,
           "offered_rate_hz": 2000.0, "rel_err_median": statistics.median(errs), "rel_err_max": max(errs),
           "slots": args.slots, "budget_gb": args.budget_gb, "prec": prec,
           "config": {"streams": n_streams, "window": list(small), "resized_window": list(big),
                      "resize_frac": 0.10, "p": p, "ranks": list(ranks), "sweeps": sweeps, "warm_start": True}}
    # one cold window (a stream with no resident state) through the server
    # against the oracle (HOSVD start + 3 sweeps)
    try:
        srv = mach.Server(int(args.budget_gb * 2 ** 30), 1)
        xc = pool[0][0]
        t = srv.submit(10 ** 6, xc, ranks, p, 4242, sweeps, prec)
        G_g, A_g, _ = _drain(srv, [t])[0]
        srv.close()
        out["oracle_check"] = oracle_checks([(xc.cpu().numpy(), ranks, p, 4242, sweeps, G_g, A_g,
                                              "cold window 200x16x512 through the server")])[0]
    except Exception as ex:  # report, never fail the line
        out["oracle_check"] = {"error": str(ex)[:300]}
    return out


ORACLE_CHECK_SNIPPET = r"""
import sys, time, json
sys.path.insert(0, %(root)r)
import numpy as np
from oracle import mach_oracle as O
X = np.load(%(xpath)r)
z = np.load(%(gpath)r)
G_g = z["G"]
A_g = [z["A%%d" %% k] for k in range(X.ndim)]
O.build_oracle_lib()
t0 = time.perf_counter()
S, G, A = O.mach_hooi(X, %(ranks)r, %(p)r, %(seed)r, %(sweeps)r)
t1 = time.perf_counter()
np.savez(%(out)r, G=G, **{"A%%d" %% k: a for k, a in enumerate(A)})
print(json.dumps({"seconds": t1 - t0, "rel_err_oracle": O.relative_error(X, G, A),
                  "rel_err_gpu": O.relative_error(X, G_g, A_g)}))
"""


def oracle_checks(jobs, parallel=None):
    """The oracle on small tensors (spawned single-threaded processes, run in
    parallel on the host cores) against GPU decompositions of them.  A job is
    (X numpy, ranks, p, seed, sweeps, G_gpu, [A_gpu], label)."""
    import numpy as np
    tmp = scratch_dir()
    out = []
    try:
        procs = []
        for j, (X, ranks, p, seed, sweeps, G_g, A_g, what) in enumerate(jobs):
            xpath, gpath, opath = (os.path.join(tmp, "%s%d.np%s" % (n, j, e))
                                   for n, e in (("x", "y"), ("g", "z"), ("o", "z")))
            np.save(xpath, np.ascontiguousarray(X))
            np.savez(gpath, G=_np(G_g), **{"A%d" % k: _np(a) for k, a in enumerate(A_g)})
            code = ORACLE_CHECK_SNIPPET % dict(root=ROOT, xpath=xpath, gpath=gpath, out=opath, ranks=tuple(ranks),
                                               p=p, seed=seed, sweeps=sweeps)
            procs.append((code, opath, G_g, A_g, what))
        par = parallel or host_cores()
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        running = []
        queue = list(procs)
        results = {}
        while queue or running:
            while queue and len(running) < par:
                code, opath, G_g, A_g, what = queue.pop(0)
                running.append((subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                                                 stderr=subprocess.PIPE, text=True, env=env), opath, G_g, A_g, what))
            pr, opath, G_g, A_g, what = running.pop(0)
            try:
                res = oracle_result(pr, timeout=1800)
                G_o, A_o = load_oracle_decomp(opath, len(A_g))
                c = compare(G_g, A_g, G_o, A_o)
                c.update({"what": what, "oracle_seconds": res["seconds"], "rel_err_oracle": res["rel_err_oracle"],
                          "rel_err_gpu": res["rel_err_gpu"],
                          "rel_err_diff": abs(res["rel_err_gpu"] - res["rel_err_oracle"])})
            except Exception as ex:
                c = {"what": what, "error": str(ex)[:300]}
            results[what] = c
        out = [results[p[4]] for p in procs]
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    return out


def batched_results(args, n=None, fp64_subset=64, oracle_subset=6):
    """512 independent FP32 tensors of uneven sizes (hosts U{50..400}, types
    U{8..32}, timeticks log-uniform 64..2048), rank (4, 4, 8), 10% noise,
    p = 0.1, 10 sweeps.  The value is the one-launch form (every tensor
    sampled, then mach_hooi_batched); beside it the served form (all
    submitted at once to the server: continuous batching over `slots`
    streams) and the plain FP64 form (one decomposition at a time, FP64
    sweeps) on the first `fp64_subset` tensors, and the oracle on the first
    `oracle_subset`."""
    import concurrent.futures as cf
    import torch
    from paper_0909_4969_gb300 import mach, synth
    n = n or args.batch
    ws = synth.config_batched(n)
    xs = [synth.tucker_torch(w.spec)[0] for w in ws]
    torch.cuda.synchronize()
    ranks = (4, 4, 8)
    prec = args.prec or "fp32"

    def run(pr, slots, items):
        srv = mach.Server(int(args.budget_gb * 2 ** 30), slots)
        t0 = time.perf_counter()
        tickets = [srv.submit(b, x, ranks, 0.1, b, 10, pr) for b, x in items]
        res = _drain(srv, tickets)
        t1 = time.perf_counter()
        st = srv.stats()
        srv.close()
        return len(items) / (t1 - t0), st, [r[2] for r in res]

    sample_streams = [torch.cuda.Stream() for _ in range(args.slots)]

    def sample_slot(j, items):
        st = sample_streams[j]
        return [(b, mach.sample(x, 0.1, b, stream=st)) for b, x in items[j::len(sample_streams)]]

    def one_launch(items, keep=False):
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
        return len(items) / (t1 - t0), errs, flags, (cores, facs)

    items = list(enumerate(xs))
    one_launch(items[:32])
    run(prec, args.slots, items[:32])
    value, errs, flags, (cores, facs) = one_launch(items)
    srv_value, st, srv_errs = run(prec, args.slots, items)
    sub = items[:min(fp64_subset, len(items))]
    plain, _, errs64 = run("fp64", 1, sub)
    out = {"value": value, "unit": "decompositions/s", "tensors": len(items),
           "form": "mach_sample per tensor (%d threads / streams) + mach_hooi_batched (one launch)" % args.slots,
           "total_input_gb": sum(x.numel() * 4 for x in xs) / 1e9,
           "rel_err_median": statistics.median(errs), "rel_err_max": max(errs), "device_flags": flags,
           "served_form": {"value": srv_value, "unit": "decompositions/s", "slots": args.slots, "prec": prec,
                           "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_in_flight": st["max_in_flight"],
                           "rel_err_median": statistics.median(srv_errs), "rel_err_max": max(srv_errs)},
           "plain_fp64": {"value": plain, "unit": "decompositions/s", "slots": 1, "tensors": len(sub),
                          "rel_err_median": statistics.median(errs64),
                          "rel_err_median_fp32_same_tensors": statistics.median(errs[:len(sub)]),
                          "rel_err_max_abs_diff_vs_fp32": max(abs(a - b) for a, b in zip(errs64, errs))}}
    jobs = [(xs[b].cpu().numpy(), ranks, 0.1, b, 10, cores[b], facs[b],
             "batched tensor %d %s" % (b, "x".join(map(str, xs[b].shape))))
            for b in range(min(oracle_subset, len(items)))]
    checks = oracle_checks(jobs)
    ok = [c for c in checks if "subspace_distance_max" in c]
    out["oracle_check"] = {"tensors": len(checks),
                           "subspace_distance_max": max((c["subspace_distance_max"] for c in ok), default=None),
                           "rel_err_diff_max": max((c["rel_err_diff"] for c in ok), default=None),
                           "items": checks}
    return out


def run_served(args):
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_0909_4969_gb300 import mach
    mach.load()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    r = served_results(args)
    clk = clocks.stop()
    line = {"metric": METRIC, "value": r["value"], "unit": "decompositions/s", "n_gpus": 1, "steps": args.requests,
            "warmup": max(32, 16 * args.warmup), "ms_per_step": 1e3 / r["value"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAME.get(r["prec"], r["prec"]),
            "data": "synthetic",
            "config": dict(r["config"], workload="served_stream_64x200x16x512", slots=args.slots,
                           budget_gb=args.budget_gb, requests=args.requests, prec=r["prec"]),
            "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"], "served": r, "clocks": clk}
    print(json.dumps(line))
    return 0


def run_batched(args):
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_0909_4969_gb300 import mach
    mach.load()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    r = batched_results(args)
    clk = clocks.stop()
    line = {"metric": METRIC, "value": r["value"], "unit": "decompositions/s", "n_gpus": 1, "steps": r["tensors"],
            "warmup": 32, "ms_per_step": 1e3 / r["value"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched_%d_uneven" % r["tensors"], "ranks": [4, 4, 8], "p": 0.1, "sweeps": 10,
                       "noise": 0.10, "form": r["form"]},
            "batched": r, "clocks": clk}
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
    import numpy as np
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
    w_r = synth.Workload(w.name, spec_r, w.p, w.sweeps, w.precision)
    X, _, _ = synth.tucker_torch(spec_r, device="cuda")
    torch.cuda.synchronize()
    # the full-size oracle (rank 0, one GPU only) runs on the host after the
    # timed region, beside the untimed-for-the-headline GPU legs; X goes to a
    # scratch file first
    oracle_job = None
    tmp = None
    want_oracle = rank == 0 and world == 1 and not args.no_cpu_baseline
    if want_oracle:
        tmp = scratch_dir()
        xpath = os.path.join(tmp, "x.npy")
        np.save(xpath, X.cpu().numpy())
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

    def step(x, pr=prec):
        s = mach.sample(x, w.p, spec_r.seed)
        if args.workload == "tucker2_sensor":
            G, A = s.tucker2((ranks[0], ranks[1], 0), 2, w.sweeps, pr)   # time mode kept whole
        else:
            G, A = s.hooi(ranks, w.sweeps, pr)
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
    if want_oracle:
        slab = args.cpu_slab if w.name.startswith("mixed_4way") else 0
        oracle_out = os.path.join(tmp, "oracle.npz")
        oracle_job = (oracle_proc(xpath, w_r, out=oracle_out, slab=slab), slab, oracle_out)
    total_ms = e0.elapsed_time(e1)
    per_step = [a.elapsed_time(b) for a, b in step_ms]
    total_ms = max_over_ranks(total_ms, world, "cuda")
    value = replica_throughput(args.steps, world, total_ms)
    eig_stats = dict(last_stats)

    # per-kernel-class profile (library-recorded CUDA events on this stream)
    prof = {}
    for kind, name in enumerate(PROF_KINDS):
        ms = mach.ctypes.c_double()
        n = mach.ctypes.c_int64()
        by = mach.ctypes.c_double()
        lib.mach_profile_query(kind, mach.ctypes.byref(ms), mach.ctypes.byref(n), mach.ctypes.byref(by))
        prof[name] = {"ms": ms.value, "launches": n.value, "bytes": by.value}
    lib.mach_profile_enable(0)
    hbm_peak, peak_kind = measured_peaks()
    step_avg = total_ms / args.steps
    shares = {k: v["ms"] / args.steps / step_avg for k, v in prof.items()}
    # the roofline kernel: the largest HBM-bound class (the sampler or the TTM
    # chain); `class_shares` gives every class's share of the step, and the
    # latency-bound classes carry no HBM or tensor roofline
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
                "avg_launch_ms": d["ms"] / max(d["launches"], 1),
                "largest_class": max(shares, key=shares.get)}

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

    # the plain FP64 GPU form of the same decomposition, timed the same way
    plain = None
    G64 = A64 = None
    if not args.no_fp64 and prec != "fp64":
        step(X, "fp64")
        torch.cuda.synchronize()
        f64 = []
        for _ in range(max(1, args.fp64_steps)):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            G64, A64 = step(X, "fp64")
            b.record(stream)
            f64.append((a, b))
        torch.cuda.synchronize()
        t64 = [a.elapsed_time(b) for a, b in f64]
        plain = {"value": 1e3 / statistics.mean(t64), "unit": "decompositions/s", "ms_per_step": statistics.mean(t64),
                 "steps": len(t64), "dtype": "f64", "eigensolver": dict(last_stats),
                 "speedup_of_timed_form": value / (1e3 / statistics.mean(t64))}

    # accuracy of the timed form (the last timed step's decomposition)
    accuracy = {}
    if args.workload != "tucker2_sensor":
        err32 = mach.error(X, G, A)[0]
        accuracy["rel_err"] = err32
        if G64 is not None:
            err64 = mach.error(X, G64, A64)[0]
            c = compare(G, A, G64, A64)
            c.update({"rel_err_fp64": err64, "rel_err_diff": abs(err32 - err64)})
            accuracy["vs_plain_fp64"] = c

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
            Ge, Ae = step(xdev)
            outs = [Ge.cpu()] + [a.cpu() for a in Ae if a is not None]
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

    # the batched and served workloads, compact (default workload only)
    sub = {}
    if rank == 0 and world == 1 and not args.no_sub and args.workload == "large_fp32":
        for name, fn in (("batched", batched_results), ("served", served_results)):
            try:
                sub[name] = fn(args)
            except Exception as ex:   # report, never fail the bench line
                sub[name] = {"error": str(ex)[:300]}

    cpu = None
    if oracle_job is not None:
        proc, slab, oracle_out = oracle_job
        try:
            res = oracle_result(proc)
            dims = list(w.spec.dims)
            if slab:
                dims[-1] = min(slab, dims[-1])
            full = not slab
            cpu = {"value": 1.0 / res["seconds"] if full else None, "unit": "decompositions/s", "cores": 1,
                   "kind": "oracle", "seconds": res["seconds"],
                   "sample": ("one whole oracle decomposition (coin, HOSVD init, %d sweeps, core) of the timed input "
                              "at full size %s (%d kept), single-threaded" %
                              (w.sweeps, "x".join(map(str, dims)), res["kept"])) if full else
                             ("oracle on the first %d of %d last-mode slices (%s, %d kept), single-threaded; "
                              "not scaled (the full tensor is too large for it)" %
                              (dims[-1], w.spec.dims[-1], "x".join(map(str, dims)), res["kept"]))}
            if full and args.workload != "tucker2_sensor":
                G_o, A_o = load_oracle_decomp(oracle_out, len(ranks))
                Gt = torch.from_numpy(G_o).cuda()
                At = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in A_o]
                e_o = mach.error(X, Gt, At)[0]
                c = compare(G, A, G_o, A_o)
                c.update({"rel_err_oracle": e_o, "rel_err_diff": abs(accuracy["rel_err"] - e_o)})
                accuracy["vs_oracle"] = c
                if G64 is not None:
                    c = compare(G64, A64, G_o, A_o)
                    c.update({"rel_err_diff": abs(accuracy["vs_plain_fp64"]["rel_err_fp64"] - e_o)})
                    accuracy["plain_fp64_vs_oracle"] = c
                accuracy["note"] = ("rel_err: Section 4's ||X - G x A|| / ||X|| against the input, all by "
                                    "mach_error; subspace distance ||A A^T - B B^T||_F / sqrt(2r); core after "
                                    "fixing column signs")
        except Exception as ex:  # report, never fail the bench line
            cpu = {"value": None, "unit": "decompositions/s", "cores": 1, "kind": "oracle", "sample": str(ex)[:300]}
    if tmp:
        shutil.rmtree(tmp, ignore_errors=True)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "decompositions/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAME.get(prec, prec),
                "data": "synthetic", "config": config_dict(w, prec),
                "p50_ms": statistics.median(per_step),
                "p99_ms": sorted(per_step)[max(0, math.ceil(0.99 * len(per_step)) - 1)],
                "plain_fp64": plain, "accuracy": accuracy,
                "sampler_gbs": samp_gbs, "sampler_frac_of_hbm": samp_gbs / hbm_peak, "sampler_skip": skip,
                "sampler_host_stream": host_stream,
                "roofline": roofline, "class_shares": shares,
                "profile_ms_per_step": {k: v["ms"] / args.steps for k, v in prof.items()},
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
                "eigensolver": eig_stats}
        line.update(sub)
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
