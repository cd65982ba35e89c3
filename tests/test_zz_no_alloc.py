"""The no-allocation entry point (phylo_evaluate_noalloc), for callers that
cannot allocate device memory: runtimes whose GPU memory belongs to their
own pool, and fixed-footprint samplers that must not grow after start-up.
Its result must agree with the workspace path (phylo_evaluate) within the
FP32 tolerances of the parity tests, on two calls in a row (the second
finds the static scratch holding the first call's contents).  Collected
last on purpose, so that a failure here stops a -x run only after every
other test has run."""
import ctypes

import numpy as np
import pytest

import synth
from parity import TOL


def _call(lib, w, V, Vi, lam, stream=None):
    N, C, S, R = w.n_tips, w.n_patterns, w.n_states, w.n_categories
    dp = lambda a: np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(
        ctypes.POINTER(ctypes.c_double))
    keep = [np.ascontiguousarray(x, dtype=np.float64)
            for x in (w.pattern_weights, V, Vi, lam, w.pi, w.rates,
                      w.weights, w.t)]
    parent = np.ascontiguousarray(w.parent, dtype=np.int32)
    states = np.ascontiguousarray(w.tip_states, dtype=np.uint8)
    logL = ctypes.c_double(0.0)
    grad = np.zeros(2 * N - 2)
    msg = ctypes.create_string_buffer(256)
    rc = lib.phylo_evaluate_noalloc(
        N, C, S, R, parent.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
        states.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
        *[k.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for k in keep],
        ctypes.byref(logL), grad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        stream, msg, 256)
    return rc, logL.value, grad, msg.value.decode()


def test_noalloc_rejects_oversized_problems():
    """Size limits are checked on the host before any CUDA call."""
    from paper_2303_04390_gb300 import build as B, _native
    B.build()
    lib = _native.load()
    V = np.eye(4)
    big = synth.small_workload(600, 4, 2, 3, seed=41)
    rc, _, _, msg = _call(lib, big, V, V, np.zeros(4))
    assert rc == -1 and "n_tips" in msg
    wide = synth.small_workload(300, 20, 8, 2000, seed=42)
    Vw = np.eye(20)
    rc, _, _, msg = _call(lib, wide, Vw, Vw, np.zeros(20))
    assert rc == -1 and "bytes of scratch" in msg


@pytest.mark.gpu
@pytest.mark.parametrize("S", [4, 20, 61])
def test_noalloc_matches_workspace_path_twice(S):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2303_04390_gb300 as pg
    from paper_2303_04390_gb300 import _native
    from oracle import phylo_oracle as O
    lib = _native.load()
    n, c = (40, 300) if S < 61 else (20, 200)  # within the 32 MiB scratch
    w1 = synth.small_workload(n, S, 4, c, seed=43)
    w2 = synth.small_workload(n, S, 4, c, seed=44)  # different inputs
    for w in (w1, w2):
        V, Vi, lam = pg.eigen_reversible(w.Q, w.pi)
        rc, logL, grad, msg = _call(lib, w, V, Vi, lam)
        assert rc == 0, msg
        ctx = pg.from_workload(w, "fp32")
        ref_ll, ref_g = ctx.evaluate()
        ctx.close()
        _, _, _, B = O.evaluate_with_scales(
            w.parent, w.t, w.Q, w.pi, w.rates, w.weights, w.pattern_weights,
            tip_states=w.tip_states)
        tol = TOL["fp32"]
        assert abs(logL - ref_ll) <= tol["ll_rel"] * abs(ref_ll)
        bound = np.maximum(tol["g_rel"] * np.abs(ref_g), tol["g_cond"] * B)
        assert np.all(np.abs(grad - ref_g) <= bound)
