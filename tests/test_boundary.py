"""CPU tests of the C-ABI boundary: the library builds, loads and exports
every symbol include/phylo_api.h declares; the host-side logic (sizes,
validation, the host FP64 eigendecomposition) behaves as documented.  No
call here reaches the GPU: every invalid input is rejected before any CUDA
call."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "phylo_api.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2303_04390_gb300 import build as B
    B.build()
    from paper_2303_04390_gb300 import _native
    return _native.load()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\w[\w\s\*]*?\b(phylo_\w+)\s*\(", text,
                                 flags=re.M)))


def test_header_declares_the_abi():
    names = declared_functions()
    assert "phylo_evaluate" in names and "phylo_create" in names
    assert len(names) >= 15


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2303_04390_gb300 import _native
    assert set(declared_functions()) <= set(_native.SIGNATURES)


def test_workspace_bytes(lib):
    from paper_2303_04390_gb300 import workspace_bytes
    b32 = workspace_bytes(1024, 10000, 4, 4, "fp32")
    b64 = workspace_bytes(1024, 10000, 4, 4, "fp64")
    # two FP32 partial buffers of (N-1) x C x R x 4 dominate
    part = 2 * 1023 * 10000 * 4 * 4 * 4
    assert part < b32 < part * 1.2
    assert b64 > 1.9 * b32 - 1e7
    assert workspace_bytes(8, 0, 4, 1, "fp64") > 0
    tp = workspace_bytes(16, 100, 20, 4, "fp32", tip_partials=True)
    assert tp - workspace_bytes(16, 100, 20, 4, "fp32") >= 16 * 100 * 20 * 4


@pytest.mark.parametrize("S, SP, per_tip", [(20, 20, None), (61, 64, None), (122, 128, None),
                                            (4, 4, 0), (61, 64, 0)])
def test_workspace_u_slots_for_tip_partials(lib, S, SP, per_tip):
    """The U-form FP32 paths (20, 64 and 128 padded states) keep U = P p of
    every tip with partials in N extra post-order slots ([C][R][S_pad] FP32
    each, tile-padded for 20 states) beside the tips' partials ([C][S_pad]);
    the 4-state path and the FP64 path form a tip's product where it is
    needed and only store the partials."""
    from paper_2303_04390_gb300 import workspace_bytes
    N, C, R = 16, 100, 4
    prec = "fp32" if per_tip is None else ("fp32" if SP == 4 else "fp64")
    grow = (workspace_bytes(N, C, S, R, prec, tip_partials=True)
            - workspace_bytes(N, C, S, R, prec))
    elem = 4 if prec == "fp32" else 8
    partials = N * C * SP * elem
    if per_tip is None:  # tip partials plus N U slots
        slots = N * C * R * SP * 4
        assert grow >= partials + slots
        assert grow < partials + 2 * slots + 65536
    else:                # tip partials only
        assert partials <= grow < partials + 65536


@pytest.mark.parametrize("args", [(1, 10, 4, 1), (8, -1, 4, 1), (8, 10, 1, 1),
                                  (8, 10, 257, 1), (8, 10, 4, 0), (8, 10, 4, 9),
                                  (70000, 10, 4, 1)])
def test_workspace_bytes_rejects_bad_sizes(lib, args):
    out = ctypes.c_size_t(0)
    rc = lib.phylo_workspace_bytes(*args, 1, 0, ctypes.byref(out))
    assert rc == -1
    assert lib.phylo_last_error(None)


def test_workspace_bytes_rejects_overflow(lib):
    out = ctypes.c_size_t(0)
    # 65536 tips x 2^31-1 patterns x 64 states x 8 categories overflows
    rc = lib.phylo_workspace_bytes(65536, 2**31 - 1, 64, 8, 0, 0,
                                   ctypes.byref(out))
    assert rc in (-1, 0)
    if rc == 0:
        assert out.value > 2**40


FAKE_WS = 1 << 40  # never dereferenced by the host-side checks below


def _ctx(lib, N=5, C=3, S=4, R=2, prec=1, flags=0, ws=FAKE_WS, nbytes=None):
    if nbytes is None:
        b = ctypes.c_size_t(0)
        assert lib.phylo_workspace_bytes(N, C, S, R, prec, flags,
                                         ctypes.byref(b)) == 0
        nbytes = b.value
    ctx = ctypes.c_void_p()
    rc = lib.phylo_create(ctypes.byref(ctx), N, C, S, R, prec, flags,
                          ctypes.c_void_p(ws), nbytes, None)
    return rc, ctx


def test_create_validates_workspace(lib):
    rc, _ = _ctx(lib, ws=FAKE_WS + 8)
    assert rc == -1 and b"aligned" in lib.phylo_last_error(None)
    rc, _ = _ctx(lib, nbytes=100)
    assert rc == -2
    rc, ctx = _ctx(lib)
    assert rc == 0
    lib.phylo_destroy(ctx)


def _ip(a):
    return np.ascontiguousarray(a, dtype=np.int32).ctypes.data_as(
        ctypes.POINTER(ctypes.c_int32))


def _dp(a):
    return np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(
        ctypes.POINTER(ctypes.c_double))


def test_set_tree_validation_cases(lib):
    rc, ctx = _ctx(lib)  # N = 5: nodes 0..8, root 8
    bad = {
        b"not an internal node": [5, 5, 6, 6, 3, 7, 7, 8, -1],
        b"more than two children": [5, 5, 5, 6, 6, 7, 7, 8, -1],
        b"the root": [5, 5, 6, 6, 7, 7, 8, 8, 0],
        b"cycle": [5, 6, 7, 8, 8, 6, 7, 5, -1],
    }
    for msg, parent in bad.items():
        assert lib.phylo_set_tree(ctx, _ip(parent)) == -1, msg
        assert msg in lib.phylo_last_error(ctx), (msg, lib.phylo_last_error(ctx))
    lib.phylo_destroy(ctx)


def test_input_validation(lib):
    rc, ctx = _ctx(lib, N=5, C=3, S=4, R=2)
    states = np.zeros((5, 3), dtype=np.uint8)
    states[2, 1] = 5  # > S (S itself is the gap code)
    assert lib.phylo_set_tip_states(
        ctx, states.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))) == -1
    assert lib.phylo_set_pattern_weights(ctx, _dp([1.0, -1.0, 2.0])) == -1
    assert lib.phylo_set_pattern_weights(ctx, _dp([1.0, np.nan, 2.0])) == -1
    assert lib.phylo_set_categories(ctx, _dp([0.5, 1.5]), _dp([0.5, 0.4])) == -1
    assert b"sum" in lib.phylo_last_error(ctx)
    assert lib.phylo_set_categories(ctx, _dp([-0.5, 1.5]), _dp([0.5, 0.5])) == -1
    t = np.full(8, 0.1)
    t[3] = -0.1
    assert lib.phylo_set_branch_lengths(ctx, ctypes.c_void_p(t.ctypes.data),
                                        0) == -1
    t[3] = np.inf
    assert lib.phylo_set_branch_lengths(ctx, ctypes.c_void_p(t.ctypes.data),
                                        0) == -1
    # tip partials need the flag
    assert lib.phylo_set_tip_partials(ctx, 0, _dp(np.ones((3, 4)))) == -1
    # evaluation before the inputs are set
    x = ctypes.c_double(0)
    assert lib.phylo_evaluate(ctx, ctypes.byref(x), None) == -4
    assert b"not set" in lib.phylo_last_error(ctx)
    lib.phylo_destroy(ctx)


def test_tip_partials_validation(lib):
    rc, ctx = _ctx(lib, N=5, C=3, S=4, R=2, flags=1)
    p = np.ones((3, 4))
    p[1] = 0.0
    assert lib.phylo_set_tip_partials(ctx, 0, _dp(p)) == -1
    p[1] = -1.0
    assert lib.phylo_set_tip_partials(ctx, 0, _dp(p)) == -1
    assert lib.phylo_set_tip_partials(ctx, 7, _dp(np.ones((3, 4)))) == -1
    lib.phylo_destroy(ctx)


def test_eigen_validation(lib):
    rc, ctx = _ctx(lib, S=4)
    Q, pi = synth.hky85(2.0, np.array([0.1, 0.2, 0.3, 0.4]))
    from paper_2303_04390_gb300 import eigen_reversible
    V, Vi, lam = eigen_reversible(Q, pi)
    Vbad = V.copy()
    Vbad[0, 0] += 1e-3
    assert lib.phylo_set_eigen(ctx, _dp(Vbad), _dp(Vi), _dp(lam), _dp(pi)) == -1
    assert lib.phylo_set_eigen(ctx, _dp(V), _dp(Vi), _dp(lam),
                               _dp(pi * 1.1)) == -1
    # non-reversible generator
    Qn = Q.copy()
    Qn[0, 1] += 0.3
    Qn[0, 0] -= 0.3
    assert lib.phylo_set_rate_matrix(ctx, _dp(Qn), _dp(pi)) == -1
    assert b"reversible" in lib.phylo_last_error(ctx)
    lib.phylo_destroy(ctx)


@pytest.mark.parametrize("S", [2, 4, 7, 20, 33, 61, 64, 122, 256])
def test_host_eigendecomposition(lib, S):
    """V diag(lambda) Vinv reproduces Q; exp via the eigenvalues matches the
    library matrix exponential; one eigenvalue is exactly 0."""
    import scipy.linalg
    from paper_2303_04390_gb300 import eigen_reversible
    rng = np.random.default_rng(S)
    if S == 61:
        Q, pi = synth.codon_gy94(2.0, 0.3, rng.dirichlet(np.ones(61)))
    else:
        Q, pi = synth.random_reversible(S, rng)
    V, Vi, lam = eigen_reversible(Q, pi)
    assert np.max(np.abs(V @ np.diag(lam) @ Vi - Q)) < 1e-12 * max(1, np.abs(Q).max())
    assert np.max(np.abs(V @ Vi - np.eye(S))) < 1e-12
    assert np.sum(lam == 0.0) == 1 and np.all(lam <= 0)
    for t in [0.01, 0.5, 3.0]:
        P = V @ np.diag(np.exp(lam * t)) @ Vi
        assert np.max(np.abs(P - scipy.linalg.expm(t * Q))) < 1e-13


def test_level_schedule_launch_count_needs_tree(lib):
    rc, ctx = _ctx(lib)
    assert lib.phylo_launches_per_evaluation(ctx) == 0
    lib.phylo_destroy(ctx)
