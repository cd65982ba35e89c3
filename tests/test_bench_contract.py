"""The bench's JSON contract on the CPU (its reference arm times the oracle,
so it runs without a GPU) and the per-phase work counts the roofline
figures divide by."""
import json
import os
import subprocess
import sys

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload",
                          "jc69-8", "--steps", "3", "--warmup", "3"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [x for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 3 and d["warmup"] == 3
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "jc69-8"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_rejects_short_warmup():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload",
                          "jc69-8", "--steps", "3", "--warmup", "1"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode != 0


def test_work_counts():
    """Bytes: post reads p of the internal children and writes p of the
    internal non-root nodes; pre reads q_k and p and writes q of internal
    children.  Flops: one 2 S^2 product per internal non-root node in the
    post-order pass, three in the pre-order pass (tips are column lookups)."""
    sys.path.insert(0, ROOT)
    import bench
    N, S, R, C = 10, 61, 4, 100
    w = synth.small_workload(N, S, R, C, seed=1)
    M = R * C * S * 4
    mats = (2 * N - 2) * R * S * S * 4
    by = bench.algorithmic_bytes(w, "fp32")
    assert by["post"] == 2 * (N - 2) * M + N * C + 8 * (N - 2) * C + mats + 8 * C
    assert by["pre"] == 3 * (N - 2) * M + N * C + 2 * mats + 8 * C + 8 * (2 * N - 2)
    assert bench.algorithmic_bytes(w, "fp64")["post"] > by["post"]
    fl = bench.algorithmic_flops(w)
    assert fl["post"] == (N - 2) * 2 * S * S * R * C
    assert fl["pre"] == 3 * fl["post"] and fl["pmat"] == 0
