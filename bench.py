#!/usr/bin/env python
"""Benchmark of the PRGD hot path on one GB300.

Headline workload: the hyperspectral-shaped completion problem (the
paper's hyperspectral-image experiment, Section 5, with a synthetic tensor
in place of the image data set, which is not available): 256 x 256 x 128,
sum of 20 separable smooth terms plus N(0, 1e-3^2) noise, TT-ranks
(1,20,20,1), 10% of the entries observed (|Omega| = 838 861).  A step is one
PRGD iteration (sampled pass over Omega, weights, weighted tangent
projection, the steepest step of Eq. (PRGD stepsize), rank-2r assembly,
TT-rounding retraction) in the MIXED mode (FP32 sampled pass, FP64 dense
stages) of a batch of B independent such problems (seeds differ), launched
as one CUDA graph, all inputs resident in device memory.  The batch's inputs
are larger than L2.

The step size: the constant form of Theorem 4.1 at the tuned scale 1.5
diverges on this workload and converges ~10x slower at 0.5 (oracle runs);
the steepest step converges, so it is this workload's policy.

Prints ONE JSON line with the headline figures plus, under `configs`, the
other workloads (the planted order-4 problem, the orthogonal cubic problem,
the tomography-shaped problem), each with its batched throughput, iterations
and time to rel.err <= 1e-6 (mixed precision against plain FP64 on the
GPU) and its error against the FP64 CPU oracle.  `--impl reference` times
the FP64 CPU oracle on the headline workload instead (the reference arm;
rank 0 only).

Multi-GPU: one process per GPU (torchrun), each solving its own replicas
(disjoint seeds); value = entries of all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Ω-entries/s & PRGD iters/s to rel.err≤1e-6 vs FP64 GPU; p50/p99 solve ms"
HEADLINE = {"workload": "hyperspectral_like", "shape": [256, 256, 128], "ranks": [1, 20, 20, 1],
            "omega": 838861, "frac": 0.10, "noise_std": 1e-3, "terms": 20, "step_rule": "steepest"}
GOLDEN = os.path.join(ROOT, "tests", "golden", "full_size_solutions.json")
L2_BYTES = 129 * 2 ** 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ttc", choices=["ttc", "reference"])
    ap.add_argument("--batch", type=int, default=32, help="headline problems per step (one CUDA graph launch)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the other workloads")
    ap.add_argument("--e2e-solves", type=int, default=2)
    ap.add_argument("--e2e-iters", type=int, default=20)
    ap.add_argument("--serve-mixed", type=int, default=512,
                    help="requests of the mixed serving stream (0: skip)")
    ap.add_argument("--serve-max-entries", type=int, default=1_000_000)
    ap.add_argument("--serve-slots", type=int, default=64)
    ap.add_argument("--serve-probe", type=int, default=128,
                    help="requests of the burst that probes the service rate (the Poisson stream runs at 70%% of it)")
    ap.add_argument("--lanes", type=int, default=1, help="headline batch split into lanes (ttc_batch_set_lanes)")
    ap.add_argument("--headline-only", action="store_true",
                    help="time the headline batch only (no tolerance runs, other workloads, end to end, serving "
                         "or CPU baseline): the command the committed ncu launch lists profile")
    ap.add_argument("--workload", default="hyperspectral_like",
                    choices=["hyperspectral_like", "orthogonal_cubic", "tomography_like", "planted_small"],
                    help="with --headline-only: the workload of the timed batch (profiling commands of the other "
                         "workloads; their step rule is the constant step)")
    a = ap.parse_args()
    if a.workload != "hyperspectral_like" and not a.headline_only:
        ap.error("--workload other than hyperspectral_like needs --headline-only")
    if a.headline_only:
        a.no_configs, a.no_cpu_baseline, a.serve_mixed = True, True, 0
    return a


_T0 = time.perf_counter()


def phase(msg):
    """Progress of the run on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.perf_counter() - _T0:7.1f} s] {msg}", file=sys.stderr, flush=True)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline); every process runs one
# problem single-threaded, so `cores` is what the run actually used.
# ---------------------------------------------------------------------------
ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, %(root)r)
import oracle as o
from paper_2501_13385_gb300 import workloads as w
P = w.hyperspectral_like(%(seed)d)
cur = P.init
times = []
t_end = time.perf_counter() + %(budget)f
for i in range(%(warm)d + %(steps)d):
    t0 = time.perf_counter()
    cur, _ = o.prgd_step(cur, P.idx, P.y, P.n, P.r, eps_rel=1.0, alpha_scale=1.5, step="adaptive")
    dt = time.perf_counter() - t0
    if i >= %(warm)d:
        times.append(dt)
    if i >= %(warm)d and time.perf_counter() > t_end:
        break
print(json.dumps({"N": P.N, "times": times}))
"""


def _one_thread_env():
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[v] = "1"
    return env


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_oracle_parallel(procs, warm, steps, budget_s):
    """The oracle on `procs` independent headline problems at once (one
    single-threaded process per host core, seeds 0..procs-1), each stopping
    after the first timed step past budget_s; returns (Omega-entries per
    second of all processes, per-process results, wall seconds)."""
    t0 = time.perf_counter()
    ps = []
    for i in range(procs):
        code = ORACLE_SNIPPET % {"root": ROOT, "seed": i, "warm": warm, "steps": steps, "budget": budget_s}
        ps.append(subprocess.Popen([sys.executable, "-c", code], env=_one_thread_env(), stdout=subprocess.PIPE,
                                   stderr=subprocess.PIPE, text=True))
    res = []
    for p in ps:
        out, err = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(f"oracle process failed: {err[-400:]}")
        res.append(json.loads(out.strip().splitlines()[-1]))
    wall = time.perf_counter() - t0
    per_proc = [r["N"] * len(r["times"]) / sum(r["times"]) for r in res]
    return sum(per_proc), res, wall


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    cores = host_cores()
    value, res, wall = run_oracle_parallel(cores, 0, max(1, min(args.steps, 3)), budget_s=45.0)
    t = [x for r in res for x in r["times"]]
    ms = 1e3 * statistics.mean(t)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Ω-entries/s", "n_gpus": args.gpus,
        "steps": min(len(r["times"]) for r in res), "warmup": 0, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(HEADLINE, precision="fp64", batch=cores, parallelism=f"{cores} host processes (CPU)"),
        "iters_per_s": cores * 1e3 / ms,
        "cpu_baseline": {"value": value, "unit": "Ω-entries/s", "cores": cores, "kind": "oracle",
                         "sample": f"{cores} headline problems in parallel, one single-threaded oracle process "
                                   f"per core, {len(t)} PRGD iterations in total ({wall:.0f} s wall)"},
        "e2e": {"value": value, "unit": "Ω-entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, v in enumerate(fl) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# algorithmic work of the sampled pass (the per-unit figures of the roofline)
# ---------------------------------------------------------------------------
def code_plan(n):
    """Packed-code layout of the coordinates (fields never straddle a 32-bit
    word): per mode (word, shift, bits), and the words per entry."""
    word, shift, plan = 0, 0, []
    for nk in n:
        bits = max(0, int(nk - 1).bit_length())
        if shift + bits > 32:
            word, shift = word + 1, 0
        plan.append((word, shift, bits))
        shift += bits
    W = word + 1
    return plan, (4 if W == 3 else W)


def table_rows(P):
    """Valid rows of the interface tables the library keeps (prefix tables
    over modes 0..j-1, j >= 2, and suffix tables over modes j..d-1, j <= d-2,
    whose modes share one code word and whose bit-indexed row count stays
    within min(2^17, max(4096, 4|Omega|)))."""
    plan, _ = code_plan(P.n)
    cap = min(1 << 17, max(4096, 4 * P.N))
    rows, m = [], P.m

    def ok(first, last):
        if plan[first][0] != plan[last][0]:
            return False
        bits = plan[last][1] + plan[last][2] - plan[first][1]
        return bits <= 17 and (1 << bits) <= cap
    for j in range(2, m):
        if not ok(0, j - 1):
            break
        rows.append(math.prod(P.n[:j]))
    for j in range(m - 2, 0, -1):
        if not ok(j, m - 1):
            break
        rows.append(math.prod(P.n[j:]))
    return rows


def rank_bucket(P):
    rmax = max(P.r)
    return 4 if rmax <= 4 else 8 if rmax <= 8 else 16 if rmax <= 16 else 32


def pass_bytes(P, chunk=1024):
    """Bytes the sampled pass must move per step for one problem: for every
    mode k, every entry's packed code (4W bytes) and FP32 value (4 bytes), one
    FP32 partial (1 + r_k r_{k+1} values) per chunk of `chunk` entries of a
    slice, and, read once, the valid rows of the interface tables (r values
    each) and the core slices (r_k r_{k+1} values each)."""
    import numpy as np
    _, W = code_plan(P.n)
    total = 0
    for k in range(P.m):
        counts = np.bincount(P.idx[:, k], minlength=P.n[k])
        chunks = int(np.sum((counts + chunk - 1) // chunk))
        total += P.N * (4 * W + 4) + chunks * (1 + P.r[k] * P.r[k + 1]) * 4
        total += P.n[k] * P.r[k] * P.r[k + 1] * 4
    rows = table_rows(P)
    total += sum(rows) * max(P.r) * 4
    return total


def dense_fmas(P, steepest=True):
    """FMAs of the dense part's slice products for one problem and FP32
    step, as the library computes them (float-float): the Grams Lam, Gam
    (upper triangles), H, Psi and N, the new cores (S C P) and, with the
    steepest step, the unit-step update cores B1 and their W-norm terms.  The
    bonds' and the Gram inverses' small FP64 factorizations are not counted
    (their time is)."""
    m, r, n = P.m, P.r, P.n
    q = [1] + [2 * r[k] for k in range(1, m)] + [1]
    tot = 0.0
    for k in range(m):
        ra, rb, qa, qb = r[k], r[k + 1], q[k], q[k + 1]
        if k < m - 1:
            tot += n[k] * (ra * ra * rb + 0.5 * rb * (rb + 1) * ra)          # Lam_{k+1}
            tot += n[k] * rb * rb * ra                                         # H_k
            tot += n[k] * ((0.5 * qb * (qb + 1) * qa) if k == 0 else (qb * ra * qa + 0.5 * qb * (qb + 1) * ra))   # N_k
        if k > 0:
            tot += n[k] * (ra * rb * rb + 0.5 * ra * (ra + 1) * rb)          # Gam_k
            tot += n[k] * (qa * qb * qb + 0.5 * qa * (qa + 1) * qb)          # Psi_k
        tot += n[k] * (ra * qb * qa + (ra * rb * qb if k < m - 1 else 0))   # new core
        if steepest:
            tot += n[k] * (ra * ra * rb + ra * rb * rb + (ra * rb * rb if k < m - 1 else 0))   # B1
            tot += n[k] * (ra * ra * rb + ra * rb * rb)                                      # <Lam B1 Gam, B1>
    return tot


def pass_flops(P):
    """FP32 FMAs the sampled pass must do per step for one problem when every
    interface is one table or core row (the case of the headline workload):
    per entry and mode k, the value l^T T_k(x) r (r_{k-1} r_k + min(r_{k-1},
    r_k) FMAs) and the rank-one update g l r^T (r_{k-1} r_k FMAs); as FLOPs
    (2 per FMA)."""
    fma = 0
    for k in range(P.m):
        a, b = P.r[k], P.r[k + 1]
        fma += P.N * (a * b + min(a, b) + a * b)
    return 2 * fma


def end_to_end(args, probs, world, B, N, torch, np, ttc, steep):
    """End to end through the public API from pinned host buffers: every step
    copies all B problems' observations and starting cores in, builds their
    layouts, runs e2e_iters batched iterations and reads the cores back."""
    from paper_2501_13385_gb300.replicas import max_over_ranks, whole_job_rate
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    idx_h = [pin(P.idx.astype(np.int32)) for P in probs]
    y_h = [pin(P.y) for P in probs]
    init_h = [[pin(c) for c in P.init] for P in probs]
    e2e_ms = []
    out_bytes = 0
    ectx = [ttc.Context(P.n, P.r, precision=ttc.PREC_MIXED, stop_rule=ttc.STOP_NONE, **steep) for P in probs]
    for rep in range(max(1, args.e2e_solves) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for c, ih, yh, ch in zip(ectx, idx_h, y_h, init_h):
            c.set_observations(ih, yh)
            c.set_cores(ch)
        with ttc.Batch(ectx) as eb:
            for _ in range(args.e2e_iters):
                eb.step()
            eb.sync()
        res_cores = [c.get_cores() for c in ectx]
        dt = 1e3 * (time.perf_counter() - t0)
        if rep > 0:                         # the first round captures graphs
            e2e_ms.append(dt)
        out_bytes = sum(a.nbytes for cs in res_cores for a in cs)
    for c in ectx:
        c.close()
    h2d = sum(a.nbytes for a in idx_h) + sum(a.nbytes for a in y_h) + sum(a.nbytes for cs in init_h for a in cs)
    e2e_step_ms = max_over_ranks(statistics.mean(e2e_ms), world)
    e2e_val = whole_job_rate(world, B, N, args.e2e_iters, e2e_step_ms)
    return {"value": e2e_val, "unit": "Ω-entries/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": out_bytes,
            "iters_per_step": args.e2e_iters, "ms_per_step": e2e_step_ms}


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def ttc_arm(args):
    rank, world, local = dist_env()
    if world > 1:
        os.environ.setdefault("CUDA_VISIBLE_DEVICES", str(local))
    import numpy as np
    import torch
    import torch.distributed as dist

    import oracle as o
    from paper_2501_13385_gb300 import build, ttc
    from paper_2501_13385_gb300 import workloads as w
    from paper_2501_13385_gb300.replicas import max_over_ranks, replica_seeds, whole_job_rate

    if world > 1:
        dist.init_process_group("gloo", rank=rank, world_size=world)
    build.build()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    tstream = torch.cuda.Stream(dev)
    sp = tstream.cuda_stream
    B = max(1, args.batch)

    def make_ctx(P, prec, stop=ttc.STOP_NONE, **kw):
        c = ttc.Context(P.n, P.r, precision=prec, stop_rule=stop, **kw)
        c.set_observations(P.idx, P.y)
        c.set_cores(P.init)
        return c

    def time_batch(probs, steps, warmup, prec=ttc.PREC_MIXED, clocks=False, lanes=1, **kw):
        """K timed batched steps on `tstream`, L2 flushed between steps when
        the batch's inputs fit in L2; returns a dict of figures.  With lanes
        (independent sub-batches that run ahead between joins) the K steps
        are timed as one region, from an event before the lanes fork to one
        after they join, and the pass and dense durations come from two
        profiled steps afterwards."""
        ctxs = [make_ctx(P, prec, **kw) for P in probs]
        batch = ttc.Batch(ctxs, stream=sp, lanes=lanes)
        if lanes > 1:
            return time_lanes(batch, ctxs, probs, steps, warmup, clocks)
        flush = None
        note = "inputs larger than L2 (no flush)"
        if sum(pass_bytes(P) for P in probs) < 4 * L2_BYTES:
            flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
            note = "flushed between timed steps (256 MB write)"
        for _ in range(warmup):
            batch.step()
        batch.sync()
        batch.profile_enable(True)
        batch.step()                          # recaptures with the timing event nodes
        batch.sync()
        batch.profile_read(reset=True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        launches0 = batch.launch_count()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(local) if clocks else None
        if clk:
            clk.__enter__()
        with torch.cuda.stream(tstream):
            for i in range(steps):
                ev[i][0].record(tstream)
                batch.step()
                ev[i][1].record(tstream)
                if flush is not None:
                    flush.zero_()
        torch.cuda.synchronize()
        if clk:
            clk.__exit__()
        if world > 1:
            dist.barrier()
        launches = batch.launch_count() - launches0
        step_ms = [a.elapsed_time(b) for a, b in ev]
        kern_ms, kern_n = batch.profile_read(reset=False)
        dense_ms, _ = batch.profile_read_dense(reset=True)
        batch.close()
        for c in ctxs:
            c.close()
        return {"step_ms": step_ms, "total_ms": sum(step_ms), "launches": launches,
                "pass_ms": kern_ms / max(kern_n, 1), "pass_launches": kern_n, "l2": note,
                "dense_ms": dense_ms / max(kern_n, 1),
                "clocks": clk.summary() if clk else None}

    def time_lanes(batch, ctxs, probs, steps, warmup, clocks):
        if sum(pass_bytes(P) for P in probs) < L2_BYTES:
            raise RuntimeError("lanes need inputs larger than L2 (no step boundary to flush at)")
        for _ in range(warmup):
            batch.step()
        batch.sync()
        launches0 = batch.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(local) if clocks else None
        if clk:
            clk.__enter__()
        with torch.cuda.stream(tstream):
            e0.record(tstream)
            for _ in range(steps):
                batch.step()
            batch.join()
            e1.record(tstream)
        torch.cuda.synchronize()
        if clk:
            clk.__exit__()
        if world > 1:
            dist.barrier()
        launches = batch.launch_count() - launches0
        total = e0.elapsed_time(e1)
        batch.profile_enable(True)
        for _ in range(3):                    # the first recaptures with the timing event nodes
            batch.step()
        batch.sync()
        kern_ms, kern_n = batch.profile_read(reset=False)
        dense_ms, _ = batch.profile_read_dense(reset=True)
        batch.close()
        for c in ctxs:
            c.close()
        return {"step_ms": [total / steps] * steps, "total_ms": total, "launches": launches,
                "pass_ms": kern_ms / max(kern_n, 1), "pass_launches": kern_n,
                "l2": f"inputs larger than L2 (no flush); {len(batch.members)} problems in lanes, timed as one region",
                "dense_ms": dense_ms / max(kern_n, 1), "clocks": clk.summary() if clk else None}

    def timed_solve(P, prec, stop, tol, max_iter, truth=None, **kw):
        """A solve from P.init through the C ABI, timed end to end on the
        host (graphs captured by an untimed first run)."""
        with make_ctx(P, prec, stop, tol=tol, max_iter=max_iter, **kw) as c:
            if truth is not None:
                c.set_truth(truth)
            c.solve()
            c.set_cores(P.init)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = c.solve()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            return res, 1e3 * dt, c.get_cores()

    def to_tol(P, step_kw, noisy):
        """Iterations and time to rel.err <= 1e-6 against the FP64 GPU
        solution: for noiseless data that solution is T* itself (checked
        to 1e-10 by the parity tests); for noisy data it is the FP64 GPU
        solve under the stop rule of the paper's noise experiment (Section 5,
        step change <= 1e-5 max(1, ||T||)), the answer the plain FP64 GPU
        PRGD gives."""
        out = {}
        if noisy:
            res, ms, ref = timed_solve(P, ttc.PREC_FP64, ttc.STOP_STEP, 1e-5, 2000, **step_kw)
            out["fp64_reference"] = {"rule": "step change <= 1e-5 max(1, ||T||)", "iters": res["iters"],
                                     "converged": res["converged"], "ms": ms}
        else:
            ref = P.truth
        for name, prec in (("mixed", ttc.PREC_MIXED), ("fp64", ttc.PREC_FP64)):
            res, ms, _ = timed_solve(P, prec, ttc.STOP_RELERR, 1e-6, 2000, truth=ref, **step_kw)
            out[name] = {"iters": res["iters"], "converged": res["converged"], "ms": ms,
                         "polish_iter": res["polish_iter"]}
        return out

    def error_vs_golden(name, P, step_kw):
        """The MIXED solve under Section 5's stop rule against the oracle's
        solution under the same rule (tests/golden/full_size_solutions.json):
        relative distance estimated on the stored sample entries."""
        gold = json.load(open(GOLDEN))[name]
        with make_ctx(P, ttc.PREC_MIXED, ttc.STOP_STEP, tol=gold["tol"], max_iter=1000, **step_kw) as c:
            res = c.solve()
            vals = c.eval(np.asarray(gold["idx"], dtype=np.int32))
        ref = gold["iterates"].get(str(res["iters"]))
        out = {"rule": "step change <= 1e-5 max(1, ||T||) (Section 5)", "iters": res["iters"],
               "oracle_iters": gold["stop"], "polish_iter": res["polish_iter"]}
        if ref is not None:
            rv = np.asarray(ref["values"])
            out["rel_dist_sampled"] = float(np.sqrt(np.sum((vals - rv) ** 2) / np.sum(rv ** 2)))
        return out

    def error_vs_live_oracle(P, step_kw, oracle_kw):
        """The MIXED solve to rel.err <= 1e-6 (vs T*) against the oracle's
        FP64 solve of the same problem to 1e-12: relative Frobenius distance."""
        with make_ctx(P, ttc.PREC_MIXED, ttc.STOP_RELERR, tol=1e-6, max_iter=500, **step_kw) as c:
            c.set_truth(P.truth)
            res = c.solve()
            got = c.get_cores()
        ref = o.solve(P.init, P.idx, P.y, P.n, P.r, truth=P.truth, eps_rel=1.0, alpha_scale=1.5, max_iter=300,
                      tol=1e-12, **oracle_kw).cores
        return {"rule": "rel.err vs T* <= 1e-6", "iters": res["iters"],
                "rel_dist": o.tt_dist(got, ref) / o.tt_norm(ref)}

    steep = {"step_rule": ttc.STEP_STEEPEST}

    # ---- the headline: batched MIXED steps of the hyperspectral-shaped workload
    phase("generating the headline workload")
    if args.workload != "hyperspectral_like":   # a profiling run of another workload
        steep = {}
    probs = [w.CONFIGS[args.workload](s) for s in replica_seeds(rank, B)]
    phase("timing the headline batch")
    N = probs[0].N
    K = args.steps
    hb = time_batch(probs, K, args.warmup, clocks=True, lanes=args.lanes, **steep)
    total_ms = max_over_ranks(hb["total_ms"], world)
    ms_per_step = total_ms / K
    value = whole_job_rate(world, B, N, K, total_ms)

    # roofline of the sampled pass (bracketed by events inside the graph)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    clock_mhz = (hb["clocks"] or {}).get("sm_max_mhz") or 2070.0
    fp32_peak = 152 * 128 * 2 * clock_mhz * 1e6 / 1e12      # FP32 SIMT: 152 SMs x 128 FMA lanes x 2
    flops = sum(pass_flops(P) for P in probs)
    achieved = flops / (hb["pass_ms"] / 1e3) / 1e12
    alg_bytes = sum(pass_bytes(P) for P in probs)
    hbm_peak = peaks.get("hbm_gbs")
    # the dominant kernels: the dense part (k_stage and the kernels between
    # the pass and the next step), all members' branches concurrent
    ff_peak = fp32_peak / 6.0      # a float-float FMA is 12 FP32 operations for 2 flops
    dflops = 2.0 * sum(dense_fmas(P, steepest=bool(steep)) for P in probs)
    dach = dflops / (hb["dense_ms"] / 1e3) / 1e12
    roof_dense = {"bound": "alu", "achieved": dach, "peak": ff_peak, "unit": "TFLOP/s", "frac": dach / ff_peak,
                  "traffic": None,
                  "kernel": "dense part of the step: k_stage (Grams, Psi, N, new cores in float-float; the bonds' "
                            "and Gram inverses' FP64 factorizations on one SM each), k_build_B1, the tangent "
                            "evaluation, k_build_C (all members' graph branches, concurrent)",
                  "kernel_ms": hb["dense_ms"], "algorithmic_flops_per_launch": dflops,
                  "peak_source": "derived: FP32 SIMT peak (152 SMs x 128 lanes x 2 x max SM clock) / 6 "
                                 "(float-float FMA = 12 FP32 operations)",
                  "step_share": hb["dense_ms"] / ms_per_step}
    roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak, "traffic": None,
            "kernel": "k_sample_project_batch<float,32,24,{first,interior,last}> (three mode-class launches, "
                      "concurrent)", "kernel_ms": hb["pass_ms"],
            "launches_timed": hb["pass_launches"], "algorithmic_flops_per_launch": flops,
            "algorithmic_bytes_per_launch": alg_bytes,
            "hbm_gbs_at_algorithmic_bytes": alg_bytes / (hb["pass_ms"] / 1e3) / 1e9,
            "hbm_peak": hbm_peak, "hbm_peak_source": "measured" if hbm_peak else "fallback",
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 FLOP x max SM clock",
            "step_share": hb["pass_ms"] / ms_per_step}

    # ---- per-result errors and time to tolerance of the headline workload
    head_tol = head_err = None
    if not args.headline_only:
        phase("headline: time to tolerance and error against the oracle")
        P0 = probs[0]
        head_tol = to_tol(P0, steep, noisy=True)
        head_err = error_vs_golden("hyperspectral_like", P0, steep)

    # ---- the other workloads
    configs = {}
    if not args.no_configs:
        # (name, maker, batch, step options, oracle options, noisy, lanes): the
        # orthogonal cubic batch runs in two lanes (its step is bound by each
        # problem's chain of small dense launches, which a second lane's pass
        # overlaps)
        specs = [
            ("planted_small", w.planted_small, 32, {}, {}, False, 1),
            ("orthogonal_cubic", w.orthogonal_cubic, 32, {}, {}, False, 2),
            ("tomography_like", w.tomography_like, 8, {}, {}, True, 1),
        ]
        for name, maker, bsz, kw, okw, noisy, lanes in specs:
            phase(f"workload {name}")
            cp = [maker(s) for s in replica_seeds(rank, bsz)]
            tb = time_batch(cp, max(5, K // 2), 3, lanes=lanes, **kw)
            cms = max_over_ranks(tb["total_ms"], world) / max(5, K // 2)
            entry = {"batch": bsz, "lanes": lanes, "omega": cp[0].N, "n": cp[0].n, "ranks": cp[0].r, "ms_per_step": cms,
                     "value": whole_job_rate(world, bsz, cp[0].N, 1, cms), "unit": "Ω-entries/s",
                     "pass_ms": tb["pass_ms"], "l2": tb["l2"],
                     "to_rel_err_1e-6": to_tol(cp[0], kw, noisy)}
            if noisy:
                entry["error_vs_oracle"] = error_vs_golden(name, cp[0], kw)
            else:
                entry["error_vs_oracle"] = error_vs_live_oracle(cp[0], kw, okw)
            configs[name] = entry

    e2e = None
    if not args.headline_only:
        phase("end to end")
        e2e = end_to_end(args, probs, world, B, N, torch, np, ttc, steep)

    # ---- the mixed serving stream
    mixed = None
    if args.serve_mixed > 0:
        phase("serving stream")
        mixed = serving_stream(args, rank, ttc, w, np)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        phase("CPU baseline (oracle)")
        cores = host_cores()
        allv, res, wall = run_oracle_parallel(cores, 0, 2, budget_s=10.0)
        cpu = {"value": allv, "unit": "Ω-entries/s", "cores": cores, "kind": "oracle",
               "sample": f"{cores} headline problems at once (hyperspectral_like seeds 0..{cores - 1}), one "
                         f"single-threaded oracle process per host core, steepest step, "
                         f"{sum(len(x['times']) for x in res)} PRGD iterations in {wall:.0f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Ω-entries/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 sampled pass + float-float slice products + f64 factorizations", "data": "synthetic",
            "config": dict(HEADLINE if args.workload == "hyperspectral_like" else {"workload": args.workload},
                           batch=B, lanes=args.lanes, precision="mixed", l2=hb["l2"],
                           parallelism="replicas" if world > 1 else "single GPU"),
            "iters_per_s": 1e3 / ms_per_step,
            "problem_iters_per_s": B * 1e3 / ms_per_step,
            "step_ms_p50": statistics.median(hb["step_ms"]),
            "step_ms_p99": sorted(hb["step_ms"])[max(0, int(math.ceil(0.99 * K)) - 1)],
            "to_rel_err_1e-6": head_tol,
            "error_vs_oracle": head_err,
            "roofline": roof_dense,
            "roofline_pass": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": hb["launches"],
            "configs": configs,
            "serving_mixed_stream": mixed,
            "clocks": hb["clocks"],
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def _request(args_tuple):
    """One request of the mixed stream (built in a worker process)."""
    seed, max_entries = args_tuple
    from paper_2501_13385_gb300 import workloads as w
    return w.random_request(seed, max_entries=max_entries)


def serving_stream(args, rank, ttc, w, np):
    """The mixed serving stream: orders 3-12, modes 4-256, interior ranks
    2-16, |Omega| log-uniform in [1e3, max_entries], each request a seeded
    Gaussian-core truth with uniform Omega, solved to rel.err <= 1e-6 vs T*
    or 500 iterations with the steepest step (the safe step for unknown
    problems: the constant step's tuned scale diverges on some of them).
    The service rate is probed by a burst of the first `serve_probe`
    requests (all submitted at once); then all requests arrive as a Poisson
    stream at 70% of that rate."""
    import multiprocessing as mp
    n = args.serve_mixed
    with mp.get_context("spawn").Pool(max(1, min(16, host_cores()))) as pool:
        reqs = pool.map(_request, [(rank * 100000 + 1000 + i, args.serve_max_entries) for i in range(n)])
    mopt = ttc.default_options(precision=ttc.PREC_MIXED, stop_rule=ttc.STOP_RELERR, tol=1e-6, max_iter=500,
                               step_rule=ttc.STEP_STEEPEST)

    def run_stream(gaps, sub=None):
        sub = reqs if sub is None else sub
        with ttc.Server(max_slots=args.serve_slots) as srv:
            t0 = time.perf_counter()
            tk = []
            for Q, gap in zip(sub, gaps):
                if gap > 0:
                    time.sleep(gap)
                tk.append(srv.submit(Q.n, Q.r, Q.idx, Q.y, Q.init, truth=Q.truth, options=mopt))
            rs = [srv.poll(t, cores=False) for t in tk]
            wall_s = time.perf_counter() - t0
            st = srv.stats()
        ok = sorted(r["latency_ms"] for r in rs if r["converged"])
        q = lambda v, f: v[min(len(v) - 1, max(0, int(np.ceil(f * len(v))) - 1))] if v else None
        return {"requests": len(rs), "wall_ms": 1e3 * wall_s, "requests_per_s": len(rs) / wall_s,
                "latency_p50_ms": q(ok, 0.5), "latency_p99_ms": q(ok, 0.99),
                "converged": len(ok),
                "not_converged": sum(1 for r in rs if r["status"] == "TTC_ENOTCONV"),
                "failed": sum(1 for r in rs if r["status"] not in ("TTC_OK", "TTC_ENOTCONV")),
                "mean_iters": float(np.mean([r["iters"] for r in rs])),
                "entry_iters_per_s": st["entry_iterations"] / wall_s, "gpu_launches": st["launches"],
                "engine_busy_ms": st["busy_ms"], "batch_rebuilds": st["rebuilds"],
                "batch_rebuild_ms": st["rebuild_ms"], "admit_ms": st["admit_ms"]}
    phase(f"serving: {len(reqs)} requests generated")
    probe = reqs[:max(1, min(len(reqs), args.serve_probe))]
    burst = run_stream([0.0] * len(probe), probe)
    phase("serving: service-rate probe done")
    prng = np.random.default_rng(7)
    rate = 0.7 * burst["requests_per_s"]
    poisson = run_stream(list(prng.exponential(1.0 / rate, len(reqs))))
    poisson["arrival_rate_per_s"] = rate
    sizes = sorted(Q.N for Q in reqs)
    return {"workload": f"random_request stream (orders 3-12, modes 4-256, ranks 2-16, |Omega| log-uniform "
                        f"1e3..{args.serve_max_entries:.0e})",
            "omega_min": sizes[0], "omega_max": sizes[-1], "omega_median": sizes[len(sizes) // 2],
            "stop": "rel.err <= 1e-6 vs T* or 500 iterations, mixed precision, steepest step",
            "latency": "submission to completion; percentiles over converged requests",
            "max_slots": args.serve_slots, "burst_probe": burst, "poisson_70pct": poisson}


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    return ttc_arm(args)


if __name__ == "__main__":
    sys.exit(main())
