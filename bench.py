#!/usr/bin/env python
"""Benchmark: branch-gradient evaluations per second on one GB300.

One step = one evaluation of log P(Y) and all 2N-2 branch-length gradient
entries from new branch lengths (the quantity an HMC leapfrog step needs):
matrices (Eq. 1) -> post-order pass (Eqs. 2-3) -> pre-order pass with the
gradient (Eqs. 4, 8) -> FP64 reductions (Eq. 7).  The default workload is
the 1,024-taxon HKY85+Gamma4 alignment with 10,000 patterns in FP32.

Printed as one JSON line:
  value      evals/s, inputs resident in HBM, one CUDA graph per step
  e2e        evals/s through the C ABI with host buffers: each step copies
             the branch lengths from pinned host memory and reads log P(Y)
             and the gradient back
  ms_per_step_stats  p10 / p50 / p90 of the per-step device times (a CUDA
             event between consecutive steps)
  roofline   the dominant kernel (the phase with the largest device time)
             against the measured HBM copy bandwidth
  fp64_path  the plain FP64 path on the same workload and GPU
  extra      every other workload (codon-128, aa-256, mmm-122, jc69-8): the
             same device measurements, phases, rooflines and FP64 path
  cpu_baseline the FP64 oracle on the host: full evaluations on all host
             cores (one worker per core over pattern blocks) and on one
             thread
  served     the continuous-batching request loop on a Poisson stream of
             independent requests (p50/p99 latency, evals/s)

--impl reference times the oracle (all host cores, full evaluations) as
the reference arm.
Under torchrun each rank runs an independent replica (weak scaling, no
collective on the data path; a MAX all-reduce of the elapsed time only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("branch-gradient evals/s & HBM GB/s vs plain FP64 GPU; "
          "served p50/p99 latency")
UNIT = "evals/s"


def _workloads():
    import synth
    return {
        "hky-1024": (synth.workload_hky_1024, "fp32"),
        "codon-128": (synth.workload_codon_128, "fp32"),
        "aa-256": (synth.workload_aa_256, "fp32"),
        "jc69-8": (synth.workload_jc69_8, "fp64"),
        "mmm-122": (synth.workload_mmm_122, "fp32"),
    }


# ---------------------------------------------------------------------------
# Algorithmic bytes per evaluation (unpadded states; what the method must
# move with partials resident in HBM).  M = R * C * S * elem bytes per node.
# ---------------------------------------------------------------------------

def algorithmic_bytes(w, precision):
    N, C, S, R = w.n_tips, w.n_patterns, w.n_states, w.n_categories
    elem = 8 if precision == "fp64" else 4
    M = R * C * S * elem
    mats = (2 * N - 2) * R * S * S * elem
    return {
        # P and dP written (and V, Vinv, lambda, t read: negligible)
        "pmat": 2 * mats,
        # read p of internal children, write p of internal non-root nodes,
        # tip states, exponents written and read, P read, pattern weights
        "post": 2 * (N - 2) * M + N * C + 2 * (N - 2) * C * 4 + mats + C * 8,
        # read q_k and p of internal children, write q of internal children,
        # tip states, P and dP read, pattern weights, gradient out
        "pre": 3 * (N - 2) * M + N * C + 2 * mats + C * 8 + (2 * N - 2) * 8,
        "reduce": (2 * N - 1) * 8,
    }


def algorithmic_flops(w, precision="fp32"):
    """Dense contractions the method needs per evaluation (2 S^2 flops per
    matrix-vector product of one pattern and category).  A tip child's
    P p is a column lookup, so in the form of Eq. 8 with dP p only internal
    non-root nodes count: post-order P p once (by the parent), pre-order
    P p, dP p and P' a.  The tensor-core form for 21..128 states (FP32)
    stores U = P p in the post-order pass and writes Eq. 8's numerator
    through dP = gamma Q P, so its pre-order pass needs P' a of every
    internal child and Q' a of every child, tips included."""
    N, C, S, R = w.n_tips, w.n_patterns, w.n_states, w.n_categories
    node = 2 * S * S * R * C
    if precision == "fp32" and 20 < S <= 128:
        return {"pmat": 0, "post": node * (N - 2),
                "pre": node * ((N - 2) + (2 * N - 2)), "reduce": 0}
    return {"pmat": 0, "post": node * (N - 2), "pre": 3 * node * (N - 2), "reduce": 0}


# ---------------------------------------------------------------------------
# Clock sampling during the timed regions
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        self.lines = []
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}",
               "--format=csv,noheader,nounits", "-lms", "50"]
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            if uuid:
                cmd += ["-i", uuid if uuid.startswith("GPU-") else "GPU-" + uuid]
        except Exception:
            pass
        self.cmd = cmd

    def start(self):
        try:
            self.proc = subprocess.Popen(self.cmd, stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() in ("active", "1"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [],
                    "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power)}


# ---------------------------------------------------------------------------
# Oracle timing (the CPU baseline and the reference arm).  The oracle runs as
# it stands: one evaluation per contiguous pattern block, each block in its
# own spawned worker process with one BLAS/OpenMP thread (the paper's CPU
# scheme: threads over pattern blocks); log P(Y) and the gradient are sums
# over patterns, so the blocks' results are summed.
# ---------------------------------------------------------------------------

_POOL_W = None


def _pool_init(name, seed, n_tips, n_patterns):
    global _POOL_W
    kw = {}
    if n_tips:
        kw["n_tips"] = n_tips
    if n_patterns:
        kw["n_patterns"] = n_patterns
    _POOL_W = _workloads()[name][0](seed, **kw)


def _pool_eval(lo, hi):
    from oracle import phylo_oracle as O
    ws = _POOL_W.with_patterns(lo, hi)
    ll, g, _ = O.evaluate(ws.parent, ws.t, ws.Q, ws.pi, ws.rates, ws.weights,
                          ws.pattern_weights, tip_states=ws.tip_states)
    return ll, g


class OraclePool:
    """n_workers spawned processes, each holding the workload; evaluate()
    runs one full evaluation (or the first n_patterns patterns) split into
    n_workers contiguous pattern blocks and returns its wall time."""

    def __init__(self, name, n_workers, seed=0, n_tips=None, n_patterns=None):
        env_keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
        old = {k: os.environ.get(k) for k in env_keys}
        for k in env_keys:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(
                n_workers, initializer=_pool_init,
                initargs=(name, seed, n_tips, n_patterns))
        finally:
            for k, v in old.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.n = n_workers

    def evaluate(self, n_patterns):
        bounds = [round(n_patterns * i / self.n) for i in range(self.n + 1)]
        jobs = [(a, b) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
        t0 = time.perf_counter()
        parts = self.pool.starmap(_pool_eval, jobs, chunksize=1)
        dt = time.perf_counter() - t0
        return dt, sum(p[0] for p in parts)

    def close(self):
        self.pool.terminate()
        self.pool.join()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(name, n_patterns, n_tips=None, repeats=3):
    """The oracle on full evaluations of the workload: on all host cores
    (median of `repeats` after one warm-up) and on one thread (one
    evaluation)."""
    cores = host_cores()
    multi = OraclePool(name, cores, n_tips=n_tips, n_patterns=None)
    try:
        multi.evaluate(n_patterns)  # warm-up (imports, first-touch)
        t_multi = statistics.median(multi.evaluate(n_patterns)[0]
                                    for _ in range(repeats))
    finally:
        multi.close()
    single = OraclePool(name, 1, n_tips=n_tips)
    try:
        t_single = single.evaluate(n_patterns)[0]
    finally:
        single.close()
    return {"value": 1.0 / t_multi, "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": f"full evaluations ({n_patterns} patterns) of the FP64 "
                      f"oracle (numpy), {cores} spawned workers with one "
                      f"thread each over contiguous pattern blocks: median "
                      f"of {repeats} after one warm-up, {t_multi:.2f} s each",
            "single_thread": {"value": 1.0 / t_single, "unit": UNIT,
                              "cores": 1,
                              "sample": f"one full evaluation on one thread, "
                                        f"{t_single:.1f} s"}}


def run_reference(args):
    """The reference arm: the oracle as it stands, on every host core (one
    worker per core over contiguous pattern blocks), each step one full
    evaluation of the workload -- or, where W + K full evaluations would
    not end within about four minutes, the first n patterns of it, n sized
    to fit and stated."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    name = args.workload
    precision = _workloads()[name][1]
    kw = {}
    if args.taxa:
        kw["n_tips"] = args.taxa
    if args.patterns:
        kw["n_patterns"] = args.patterns
    C = _workloads()[name][0](0, **kw).n_patterns
    cores = host_cores()
    pool = OraclePool(name, cores, n_tips=args.taxa, n_patterns=args.patterns)
    try:
        t_cal, _ = pool.evaluate(C)  # also the first warm-up step
        budget = 240.0
        n = C
        if t_cal * (args.steps + args.warmup) > budget:
            n = max(cores, int(C * budget / (t_cal * (args.steps + args.warmup))))
        for _ in range(args.warmup - 1):
            pool.evaluate(n)
        times = [pool.evaluate(n)[0] for _ in range(args.steps)]
    finally:
        pool.close()
    total = sum(times)
    value = args.steps * (n / C) / total
    what = (f"each step one full evaluation ({C} patterns)" if n == C else
            f"each step one evaluation of the first {n} of {C} patterns "
            f"(a full evaluation takes {t_cal:.1f} s), rate scaled by {n}/{C}")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, "precision_of_our_arm": precision},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores,
                         "kind": "oracle",
                         "sample": f"{what}; FP64 oracle (numpy), {cores} "
                                   f"spawned workers with one thread each "
                                   f"over contiguous pattern blocks; step "
                                   f"times median {statistics.median(times):.2f}"
                                   f" s"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------

def _profile_record(kernel_phase, workload, precision):
    """The '- key: value' lines of the committed ncu summary of a phase's
    kernel, if it was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles",
                        f"{kernel_phase}_{workload}_{precision}.md")
    if not os.path.exists(path):
        return None
    rec = {}
    for line in open(path):
        if ":" in line and line.startswith("- "):
            k, v = line[2:].split(":", 1)
            rec[k.strip()] = v.strip()
    if rec.get("kernel_source_sha256") != kernel_source_hash():
        return None
    return rec


def _traffic_record(kernel_phase, workload, precision):
    """dram bytes per launch from the committed ncu summary (or None)."""
    rec = _profile_record(kernel_phase, workload, precision)
    try:
        return float(rec["dram_bytes_per_launch"]), int(rec["launches"])
    except (KeyError, ValueError, TypeError):
        return None


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2303_04390_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")) and f != "phylo_api.cu":
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()


def run_served(args, seed=0):
    """Served streams over a pool of distinct seeded problems (Yule trees
    with 16-2,048 taxa, 100-20,000 patterns, 4 or 20 states):
      one-shot  -- every request a new problem: first all at once (closed
                   loop, throughput mu), then a Poisson stream at 0.7 mu;
      sessions  -- HMC-like chains, each a session on one problem whose
                   next step (new branch lengths) is submitted when the
                   previous result returns; the context stays resident.
    Beside them, the requests' device times measured alone, one at a time
    (their sum over the one-shot stream's elapsed time says how much the
    concurrent streams overlap)."""
    import numpy as np
    import synth
    import torch
    import paper_2303_04390_gb300 as pg
    from paper_2303_04390_gb300.serve import (Request, Server, latency_summary,
                                              poisson_arrivals)
    pool = [synth.served_request(k, seed) for k in range(args.serve_pool)]
    n = args.serve_requests
    reqs = [pool[k % len(pool)] for k in range(n)]
    budget = int(args.serve_budget_gb * (1 << 30))
    srv = Server(memory_budget_bytes=budget, max_active=32, n_streams=16,
                 setup_workers=6)
    srv.run(reqs[:min(n, 2 * len(pool))])  # warm-up: every pool entry
    n_closed = min(n, 1024)
    t0 = time.perf_counter()
    res = srv.run(reqs[:n_closed])
    closed = latency_summary(res, time.perf_counter() - t0)
    rate = 0.7 * closed["evals_per_s"]
    arrivals = poisson_arrivals(n, rate, seed=seed + 1)
    t0 = time.perf_counter()
    res = srv.run(reqs, arrivals)
    open_s = time.perf_counter() - t0
    open_loop = latency_summary(res, open_s)
    # -- sessions: closed-loop chains, each submitting its next step ------
    n_chains = min(args.serve_chains, len(pool))
    n_steps = args.serve_chain_steps
    rng = np.random.default_rng(seed + 2)
    owner, done = {}, [0] * n_chains

    def step_t(k):
        w = pool[k]
        return w.t * np.exp(0.05 * rng.standard_normal(w.t.shape))

    def follow(rid, result):
        k = owner[rid]
        done[k] += 1
        if done[k] < n_steps:
            owner[len(owner)] = k
            return Request(pool[k], t=step_t(k), session=k)
        return None

    first = []
    for k in range(n_chains):
        owner[k] = k
        first.append(Request(pool[k], t=step_t(k), session=k))
    srv.run(first[:n_chains])  # set the sessions up (not timed)
    owner, done = {k: k for k in range(n_chains)}, [0] * n_chains
    first = [Request(pool[k], t=step_t(k), session=k) for k in range(n_chains)]
    t0 = time.perf_counter()
    res_s = srv.run(first, follow_up=follow)
    sessions = latency_summary(res_s, time.perf_counter() - t0)
    hits = sum(r.session_hit for r in res_s)
    peak_used, peak_active = srv.admission.peak_used, srv.admission.peak_active
    evictions = srv.evictions  # (close() below releases the sessions)
    srv.close()
    # -- device time of each problem alone (graph replay, events) ---------
    alone_ms = []
    for w in pool:
        ctx = pg.from_workload(w, "fp32")
        ctx.evaluate_device()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            ctx.evaluate_device()
        e1.record()
        torch.cuda.synchronize()
        alone_ms.append(e0.elapsed_time(e1) / 3)
        ctx.close()
    alone_sum_s = sum(alone_ms[k % len(pool)] for k in range(n)) / 1e3
    return {
        "requests": n, "distinct_problems": len(pool),
        "arrival": f"Poisson at 0.7 x closed-loop throughput "
                   f"({rate:.1f}/s)",
        "evals_per_s": open_loop["evals_per_s"],
        "p50_ms": open_loop["p50_ms"], "p99_ms": open_loop["p99_ms"],
        "max_ms": open_loop["max_ms"], "failed": open_loop["failed"],
        "closed_loop_evals_per_s": closed["evals_per_s"],
        "closed_loop_p50_ms": closed["p50_ms"],
        "closed_loop_p99_ms": closed["p99_ms"],
        "device_s_alone_sum": alone_sum_s,
        "open_loop_elapsed_s": open_s,
        "sessions": {
            "chains": n_chains, "steps_per_chain": n_steps,
            "arrival": "closed loop per chain: the next step (new branch "
                       "lengths) is submitted when the previous result returns",
            "evals_per_s": sessions["evals_per_s"], "p50_ms": sessions["p50_ms"],
            "p99_ms": sessions["p99_ms"], "max_ms": sessions["max_ms"],
            "failed": sessions["failed"], "session_hits": hits,
            "evictions": evictions,
        },
        "budget_gb": args.serve_budget_gb,
        "peak_resident_gb": peak_used / (1 << 30),
        "peak_active": peak_active,
    }


def _percentiles(ms_list):
    a = sorted(ms_list)

    def q(f):
        if not a:
            return None
        x = f * (len(a) - 1)
        lo = int(math.floor(x))
        hi = min(lo + 1, len(a) - 1)
        return a[lo] + (a[hi] - a[lo]) * (x - lo)
    return {"p10": q(0.1), "p50": q(0.5), "p90": q(0.9)}


class Measure:
    """Times one workload on the device: K steps after W warm-up steps, each
    step new branch lengths (already on the device) and one evaluation,
    with a CUDA event between consecutive steps on the launching stream;
    then the four phases over up to 200 more evaluations."""

    def __init__(self, pg, w, precision, stream, seed):
        import numpy as np
        import torch
        self.torch = torch
        self.w, self.precision, self.stream = w, precision, stream
        self.ctx = pg.from_workload(w, precision, stream=stream)
        self.nb = 2 * w.n_tips - 2
        self.rng = np.random.default_rng(seed)
        self.out = torch.empty(2 * w.n_tips - 1, dtype=torch.float64,
                               device="cuda")

    def branch_lengths(self, n):
        import numpy as np
        t = self.w.t[None, :] * np.exp(
            0.05 * self.rng.standard_normal((n, self.nb)))
        return t, self.torch.tensor(t, dtype=self.torch.float64, device="cuda")

    def steps(self, K, W, barrier):
        torch = self.torch
        _, t_dev = self.branch_lengths(K + W)
        for i in range(W):
            self.ctx.set_branch_lengths(t_dev[i])
            self.ctx.evaluate_device(self.out)
        self.ctx.check()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
        barrier()
        evs[0].record(self.stream)
        for i in range(K):
            self.ctx.set_branch_lengths(t_dev[W + i])
            self.ctx.evaluate_device(self.out)
            evs[i + 1].record(self.stream)
        barrier()
        self.ctx.check()
        per = [evs[i].elapsed_time(evs[i + 1]) for i in range(K)]
        return evs[0].elapsed_time(evs[K]), per

    def phases(self, n_ev, barrier):
        torch = self.torch
        _, t_dev = self.branch_lengths(n_ev)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)]
               for _ in range(n_ev)]
        barrier()
        for i in range(n_ev):
            self.ctx.set_branch_lengths(t_dev[i])
            self.ctx.evaluate_device_timed(evs[i], self.out)
        barrier()
        self.ctx.check()
        ms = [0.0] * 4
        for e in evs:
            for p in range(4):
                ms[p] += e[p].elapsed_time(e[p + 1])
        return [x / n_ev for x in ms]

    def close(self):
        self.ctx.close()


def fp64_path(pg, w, stream, K, barrier):
    """The plain FP64 path on the same workload: K timed steps."""
    m = Measure(pg, w, "fp64", stream, seed=77)
    try:
        ms, per = m.steps(K, 3, barrier)
    finally:
        m.close()
    by64 = algorithmic_bytes(w, "fp64")
    return {"value": K / (ms / 1e3), "unit": UNIT, "steps": K,
            "ms_per_step": _percentiles(per),
            "hbm_gbs_all_phases": sum(by64.values()) / (ms / K / 1e3) / 1e9}


def rooflines(w, precision, phase_ms, level_counts, peaks, n_sm, workload):
    """The dominant phase against its bound: HBM for 4 and 20 states (with
    the FP32 ALU rate beside it at 20 states), the tensor pipe for the
    tensor-core path (21-64 states, FP32; the HBM figure is the main
    roofline there too), the FP32 (FP64) ALU rate for 65-256 states."""
    hbm_peak = peaks.get("hbm_gbs")
    peak_kind = "measured" if hbm_peak else "fallback"
    hbm_peak = hbm_peak or 6800.0
    by = algorithmic_bytes(w, precision)
    fl = algorithmic_flops(w, precision)
    names = ["pmat", "post", "pre", "reduce"]
    kernels = {"pmat": "pmat_kernel", "post": "post-order level kernel",
               "pre": "pre-order level kernel (fused gradient)",
               "reduce": "reduce_kernel"}
    if precision == "fp32" and 20 < w.n_states <= 64:
        kernels = {"pmat": "pmat_tc_kernel", "post": "post_u_kernel + root_u_kernel",
                   "pre": "pre_u_kernel + ratio_tc_kernel",
                   "reduce": "reduce_kernel"}
    if precision == "fp32" and 64 < w.n_states <= 128:
        kernels = {"pmat": "pmat_big_df_kernel (writes the split operand blocks)",
                   "post": "post_tcb_kernel + root_tcb_kernel",
                   "pre": "pre_tcb_kernel + ratio_tc_kernel",
                   "reduce": "reduce_kernel"}
    phases = {}
    for n_, ms_ in zip(names, phase_ms):
        phases[n_] = {"ms": ms_, "algorithmic_bytes": by[n_],
                      "achieved_gbs": by[n_] / (ms_ / 1e3) / 1e9 if ms_ > 0 else None}
    dom = max(names, key=lambda n_: phases[n_]["ms"])
    n_launch_dom = {"pmat": 1, "reduce": 1}.get(dom)
    if n_launch_dom is None:
        n_launch_dom = level_counts[0 if dom == "post" else 1]
    achieved = phases[dom]["achieved_gbs"]
    tr = _traffic_record(dom, workload, precision)
    traffic = tr[0] if tr is not None else None
    mhz = peaks.get("sm_max_mhz") or 2070.0
    alu_peak = n_sm * 128 * 2 * mhz * 1e6 / 1e12
    alu_kind = f"derived: {n_sm} SMs x 128 FP32 lanes x 2 flop x {mhz:.0f} MHz"
    roofline = {
        "bound": "hbm", "kernel": kernels[dom], "achieved": achieved,
        "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
        "peak_kind": f"{peak_kind} (HBM copy, burst)",
        "traffic": traffic,
        "algorithmic_bytes_per_launch": by[dom] / n_launch_dom,
        "launches_per_evaluation": n_launch_dom,
        "avg_launch_ms": phases[dom]["ms"] / n_launch_dom,
    }
    if 4 < w.n_states <= 20 and precision == "fp32":
        aach = fl[dom] / (phases[dom]["ms"] / 1e3) / 1e12
        roofline["alu"] = {"achieved": aach, "peak": alu_peak, "unit": "TFLOP/s",
                           "frac": aach / alu_peak, "peak_kind": alu_kind,
                           "algorithmic_flops_per_launch": fl[dom] / n_launch_dom}
    tensor_path = precision == "fp32" and 20 < w.n_states <= 128
    if w.n_states > 64 and not tensor_path:
        if precision == "fp32":
            apeak, akind = alu_peak, alu_kind
        else:
            apeak, akind = 1.25, "nominal FP64 rate"
        aach = fl[dom] / (phases[dom]["ms"] / 1e3) / 1e12
        roofline = {
            "bound": "alu", "kernel": kernels[dom], "achieved": aach, "peak": apeak,
            "unit": "TFLOP/s", "frac": aach / apeak, "peak_kind": akind,
            "traffic": traffic,
            "algorithmic_flops_per_launch": fl[dom] / n_launch_dom,
            "launches_per_evaluation": n_launch_dom,
            "avg_launch_ms": phases[dom]["ms"] / n_launch_dom,
            "hbm": {"achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak,
                    "algorithmic_bytes_per_launch": by[dom] / n_launch_dom},
        }
    tensor = None
    if tensor_path:
        tpeak = peaks.get("bf16_tflops_sustained")
        tkind = "measured" if tpeak else "fallback"
        tpeak = tpeak or 1700.0
        tach = fl[dom] / (phases[dom]["ms"] / 1e3) / 1e12
        rec = _profile_record(dom, workload, precision) or {}
        tensor = {
            "bound": "tensor", "kernel": kernels[dom], "achieved": tach,
            "peak": tpeak, "unit": "TFLOP/s", "frac": tach / tpeak,
            "peak_kind": f"{tkind} (BF16 dense, sustained)",
            "algorithmic_flops_per_launch": fl[dom] / n_launch_dom,
            "tensor_pipe_active_pct_ncu": (float(rec["tensor_pipe_active_pct"])
                                           if "tensor_pipe_active_pct" in rec
                                           else None),
        }
    return roofline, tensor, phases, sum(by.values())


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
    from paper_2303_04390_gb300 import build as B
    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        dist.barrier()
    import paper_2303_04390_gb300 as pg

    make, default_prec = _workloads()[args.workload]
    precision = args.precision or default_prec
    kw = {}
    if args.taxa:
        kw["n_tips"] = args.taxa
    if args.patterns:
        kw["n_patterns"] = args.patterns
    w = make(rank, **kw)  # independent replica per rank
    stream = torch.cuda.current_stream()
    K, W = args.steps, args.warmup
    nb = 2 * w.n_tips - 2

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        if world > 1:
            tt = torch.tensor([x], dtype=torch.float64, device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            x = float(tt.item())
        return x

    m = Measure(pg, w, precision, stream, seed=1000 + rank)
    if args.profile:
        # profiler target: W warm-up and K evaluations, nothing else
        m.steps(K, W, barrier)
        m.close()
        return
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.2)
    # -- headline: device-resident inputs, one graph per evaluation --------
    ms, per_step = m.steps(K, W, barrier)
    ms = max_over_ranks(ms)
    value = world * K / (ms / 1e3)
    launches = m.ctx.launches_per_evaluation()
    level_counts = m.ctx.level_counts()
    # -- per-phase device times (four graph launches, events between) -----
    phase_ms = m.phases(min(max(K, 20), 200), barrier)
    # -- end to end through the C ABI with host buffers -------------------
    t_all, _ = m.branch_lengths(K + 3)
    t_host = torch.tensor(t_all, dtype=torch.float64).pin_memory()
    ll_host = torch.empty(1, dtype=torch.float64).pin_memory()
    g_host = torch.empty(nb, dtype=torch.float64).pin_memory()
    for i in range(3):
        m.ctx.set_branch_lengths(t_host[i])
        m.ctx.evaluate_into(ll_host, g_host)
    n_e2e = K
    barrier()
    t0 = time.perf_counter()
    for i in range(n_e2e):
        m.ctx.set_branch_lengths(t_host[3 + i])
        m.ctx.evaluate_into(ll_host, g_host)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e_value = world * n_e2e / e2e_s
    sampler.stop()
    clocks = sampler.summary()
    m.close()

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    roofline, tensor, phases, bytes_all = rooflines(
        w, precision, phase_ms, level_counts, peaks, n_sm, args.workload)

    # -- the plain FP64 path on the same workload (>= 20 steps) -----------
    fp64 = None
    if precision != "fp64" and not args.skip_fp64:
        fp64 = fp64_path(pg, w, stream, max(20, min(K, 100)), barrier)

    # -- every other workload: the same measurements, in 'extra' ----------
    extra = {}
    if not args.skip_extras and not (args.taxa or args.patterns):
        for name, (mk, prec) in _workloads().items():
            if name == args.workload:
                continue
            wx = mk(rank)
            mx = Measure(pg, wx, prec, stream, seed=2000 + rank)
            try:
                msx, perx = mx.steps(max(K, 20), max(W, 3), barrier)
                kx = max(K, 20)
                phx = mx.phases(min(max(K, 20), 200), barrier)
                lcx = mx.ctx.level_counts()
            finally:
                mx.close()
            rx, tx, phsx, _ = rooflines(wx, prec, phx, lcx, peaks, n_sm, name)
            ent = {"value": world * kx / (max_over_ranks(msx) / 1e3),
                   "unit": UNIT, "steps": kx, "precision": prec,
                   "taxa": wx.n_tips, "patterns": wx.n_patterns,
                   "states": wx.n_states, "categories": wx.n_categories,
                   "ms_per_step": _percentiles(perx),
                   "us_per_eval": msx / kx * 1e3,
                   "phases_ms": {k_: v_["ms"] for k_, v_ in phsx.items()},
                   "roofline": rx, "tensor_roofline": tx}
            if prec != "fp64" and not args.skip_fp64:
                ent["fp64_path"] = fp64_path(pg, wx, stream, 20, barrier)
            extra[name] = ent

    if rank != 0:
        return
    served = None
    if not args.skip_serve:
        served = run_served(args)
    cpu = None
    if world == 1 and not args.skip_cpu:
        cpu = cpu_baseline(args.workload, w.n_patterns, n_tips=args.taxa)
    s_pad = 4 if w.n_states <= 4 else 20 if w.n_states <= 20 else 64
    part_bytes = 2 * (w.n_tips - 1) * w.n_patterns * w.n_categories * \
        s_pad * (8 if precision == "fp64" else 4)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": K, "warmup": W, "ms_per_step": ms / K,
        "ms_per_step_stats": _percentiles(per_step),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if precision == "fp64" else "f32",
        "data": "synthetic",
        "config": {
            "workload": args.workload, "taxa": w.n_tips,
            "patterns": w.n_patterns, "states": w.n_states,
            "categories": w.n_categories, "precision": precision,
            "l2": f"inputs larger than L2: {part_bytes / 1e9:.2f} GB of "
                  f"partials streamed per evaluation",
            "parallelism": f"replicas x{world}",
        },
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": nb * 8,
                "d2h_bytes_per_step": (2 * w.n_tips - 1) * 8 + 8,
                "steps": n_e2e},
        "gpu_launches": K * launches,
        "launches_per_step": launches,
        "roofline": roofline,
        "tensor_roofline": tensor,
        "phases": phases,
        "hbm_gbs_all_phases": bytes_all / (ms / K / 1e3) / 1e9,
        "fp64_path": fp64,
        "extra": extra,
        "served": served,
        "cpu_baseline": cpu,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="hky-1024",
                    choices=["hky-1024", "codon-128", "aa-256", "jc69-8", "mmm-122"])
    ap.add_argument("--precision", default=None, choices=[None, "fp32", "fp64"])
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--taxa", type=int, default=None,
                    help="override the workload's number of tips")
    ap.add_argument("--patterns", type=int, default=None,
                    help="override the workload's number of patterns")
    ap.add_argument("--skip-serve", action="store_true")
    ap.add_argument("--skip-extras", action="store_true",
                    help="time the chosen workload only (no 'extra' entries)")
    ap.add_argument("--serve-requests", type=int, default=4096)
    ap.add_argument("--serve-pool", type=int, default=96)
    ap.add_argument("--serve-budget-gb", type=float, default=32.0)
    ap.add_argument("--serve-chains", type=int, default=64,
                    help="sessions (HMC-like chains) in the session stream")
    ap.add_argument("--serve-chain-steps", type=int, default=16)
    ap.add_argument("--profile", action="store_true",
                    help="run warm-up + K evaluations only (profiler target)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
