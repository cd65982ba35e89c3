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
    post-order pass, three in the pre-order pass (tips are column lookups),
    or on the tensor-core form one per internal child and one per child."""
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
    fl = bench.algorithmic_flops(w, "fp64")
    assert fl["post"] == (N - 2) * 2 * S * S * R * C
    assert fl["pre"] == 3 * fl["post"] and fl["pmat"] == 0
    # the FP32 tensor-core form: P' a of every internal child and Q' a of
    # every child (tips included) in the pre-order pass
    tc = bench.algorithmic_flops(w, "fp32")
    assert tc["post"] == fl["post"]
    assert tc["pre"] == ((N - 2) + (2 * N - 2)) * 2 * S * S * R * C


def test_percentiles():
    sys.path.insert(0, ROOT)
    import bench
    q = bench._percentiles([float(x) for x in range(11)])
    assert q == {"p10": 1.0, "p50": 5.0, "p90": 9.0}


def test_oracle_pool_blocks_sum_to_the_full_evaluation():
    """The CPU baseline's pattern-block split: the blocks' log-likelihoods
    sum to the oracle's full-workload value, and the baseline reports the
    cores it used."""
    sys.path.insert(0, ROOT)
    import bench
    from oracle import phylo_oracle as O
    w = synth.workload_jc69_8(0)
    ll, _, _ = O.evaluate(w.parent, w.t, w.Q, w.pi, w.rates, w.weights,
                          w.pattern_weights, tip_states=w.tip_states)
    pool = bench.OraclePool("jc69-8", 3)
    try:
        dt, ll_blocks = pool.evaluate(w.n_patterns)
    finally:
        pool.close()
    assert dt > 0 and abs(ll_blocks - ll) <= 1e-10 * abs(ll)
    cpu = bench.cpu_baseline("jc69-8", w.n_patterns, repeats=1)
    assert cpu["cores"] == bench.host_cores() and cpu["value"] > 0
    assert cpu["single_thread"]["cores"] == 1
