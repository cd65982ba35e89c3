"""Pattern-count scaling sweep (the synthetic analogue of the paper's
speed-up-versus-pattern-count study, Results) with a per-phase time
breakdown in the spirit of its per-kernel table (Supplementary Table S1).

    python -m paper_2303_04390_gb300.sweep [--workload codon-128]
        [--patterns 1,4,16,...] [--steps 50] [--warmup 5]

For each pattern count C the named workload is regenerated with C unique
patterns (same tree and model), evaluated `steps` times after `warmup`
untimed evaluations, and one line is printed: C, evaluations/s, patterns x
evaluations/s, and the mean device time of each phase (matrix build,
post-order pass, pre-order pass with the gradient, final reduction) from
the library's per-phase events.  Device-resident inputs, CUDA-event timing
on the context's stream.
"""
from __future__ import annotations

import argparse
import json

import torch

import synth

from .context import from_workload

_MAKERS = {
    "codon-128": synth.workload_codon_128,
    "hky-1024": synth.workload_hky_1024,
    "aa-256": synth.workload_aa_256,
    "mmm-122": synth.workload_mmm_122,
}
_PHASES = ("pmat", "post", "pre", "reduce")


def sweep_point(make, n_patterns: int, steps: int, warmup: int, precision: str = "fp32"):
    w = make(n_patterns=n_patterns)
    stream = torch.cuda.Stream()
    ctx = from_workload(w, precision, stream=stream)
    out = torch.empty(2 * w.n_tips - 1, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            ctx.evaluate_device(out)
        ctx.check()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            ctx.evaluate_device(out)
        ev1.record(stream)
        ev1.synchronize()
        total_ms = ev0.elapsed_time(ev1) / steps
        events = [torch.cuda.Event(enable_timing=True) for _ in range(len(_PHASES) + 1)]
        acc = [0.0] * len(_PHASES)
        for _ in range(steps):
            ctx.evaluate_device_timed(events, out)
            events[-1].synchronize()
            for i in range(len(_PHASES)):
                acc[i] += events[i].elapsed_time(events[i + 1])
    ctx.check()
    ctx.close()
    return {
        "patterns": w.n_patterns,
        "evals_per_s": 1e3 / total_ms,
        "pattern_evals_per_s": w.n_patterns * 1e3 / total_ms,
        "phase_ms": {p: acc[i] / steps for i, p in enumerate(_PHASES)},
    }


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", default="codon-128", choices=sorted(_MAKERS))
    ap.add_argument("--patterns", default="1,4,16,64,256,1024,2048,4096,8192,16384")
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    args = ap.parse_args(argv)
    for c in [int(x) for x in args.patterns.split(",")]:
        rec = sweep_point(_MAKERS[args.workload], c, args.steps, args.warmup, args.precision)
        rec["workload"] = args.workload
        rec["precision"] = args.precision
        print(json.dumps(rec), flush=True)


if __name__ == "__main__":
    main()
