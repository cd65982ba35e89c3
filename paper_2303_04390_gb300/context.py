"""Python handle over one libphylograd context.

PyTorch supplies the device workspace (caching allocator) and the stream;
the library does all the work.  Method names follow the C ABI
(``phylo_set_tree`` -> ``set_tree`` ...).
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import _native as N


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def workspace_bytes(n_tips, n_patterns, n_states, n_categories,
                    precision="fp32", tip_partials=False) -> int:
    lib = N.load()
    out = ctypes.c_size_t(0)
    rc = lib.phylo_workspace_bytes(
        n_tips, n_patterns, n_states, n_categories, _prec(precision),
        N.PHYLO_FLAG_TIP_PARTIALS if tip_partials else 0, ctypes.byref(out))
    N.check(rc)
    return int(out.value)


def eigen_reversible(Q: np.ndarray, pi: np.ndarray):
    """Host FP64 eigendecomposition of a reversible Q (the library's)."""
    lib = N.load()
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    pi = np.ascontiguousarray(pi, dtype=np.float64)
    S = Q.shape[0]
    V = np.zeros((S, S))
    Vi = np.zeros((S, S))
    lam = np.zeros(S)
    N.check(lib.phylo_eigen_reversible(S, _dptr(Q), _dptr(pi), _dptr(V),
                                       _dptr(Vi), _dptr(lam)))
    return V, Vi, lam


def _prec(p) -> int:
    if p in ("fp64", N.PHYLO_FP64):
        return N.PHYLO_FP64
    if p in ("fp32", N.PHYLO_FP32):
        return N.PHYLO_FP32
    raise ValueError(f"unknown precision {p!r}")


class PhyloContext:
    """One problem shape (N tips, C patterns, S states, R categories) with
    its inputs resident on the GPU."""

    def __init__(self, n_tips: int, n_patterns: int, n_states: int,
                 n_categories: int, precision="fp32", tip_partials=False,
                 device=None, stream=None, use_graph=True):
        import torch
        self._lib = N.load()
        self.n_tips, self.n_patterns = n_tips, n_patterns
        self.n_states, self.n_categories = n_states, n_categories
        self.precision = precision
        self.device = torch.device(device if device is not None else "cuda")
        nbytes = workspace_bytes(n_tips, n_patterns, n_states, n_categories,
                                 precision, tip_partials)
        self.workspace_nbytes = nbytes
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8,
                               device=self.device)
        base = self._ws.data_ptr()
        ptr = (base + 255) // 256 * 256
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        ctx = ctypes.c_void_p()
        flags = (N.PHYLO_FLAG_TIP_PARTIALS if tip_partials else 0) | \
            (0 if use_graph else N.PHYLO_FLAG_NO_GRAPH)
        rc = self._lib.phylo_create(
            ctypes.byref(ctx), n_tips, n_patterns, n_states, n_categories,
            _prec(precision), flags, ctypes.c_void_p(ptr), nbytes,
            ctypes.c_void_p(sp))
        N.check(rc)
        self._ctx = ctx
        self._out = None

    # -- inputs -------------------------------------------------------------
    def _check(self, rc):
        N.check(rc, self._ctx)

    def set_tree(self, parent: np.ndarray):
        p = np.ascontiguousarray(parent, dtype=np.int32)
        assert p.shape == (2 * self.n_tips - 1,)
        self._check(self._lib.phylo_set_tree(
            self._ctx, p.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))

    def set_tip_states(self, states: np.ndarray):
        s = np.ascontiguousarray(states, dtype=np.uint8)
        assert s.shape == (self.n_tips, self.n_patterns)
        self._check(self._lib.phylo_set_tip_states(
            self._ctx, s.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))

    def set_tip_partials(self, tip: int, partials: np.ndarray):
        a = np.ascontiguousarray(partials, dtype=np.float64)
        assert a.shape == (self.n_patterns, self.n_states)
        self._check(self._lib.phylo_set_tip_partials(self._ctx, tip, _dptr(a)))

    def set_pattern_weights(self, w: np.ndarray):
        a = np.ascontiguousarray(w, dtype=np.float64)
        assert a.shape == (self.n_patterns,)
        self._check(self._lib.phylo_set_pattern_weights(self._ctx, _dptr(a)))

    def set_rate_matrix(self, Q: np.ndarray, pi: np.ndarray):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        pi = np.ascontiguousarray(pi, dtype=np.float64)
        self._check(self._lib.phylo_set_rate_matrix(self._ctx, _dptr(Q),
                                                    _dptr(pi)))

    def set_eigen(self, V, Vinv, lam, pi):
        arrs = [np.ascontiguousarray(x, dtype=np.float64)
                for x in (V, Vinv, lam, pi)]
        self._check(self._lib.phylo_set_eigen(self._ctx,
                                              *[_dptr(x) for x in arrs]))

    def set_categories(self, rates: np.ndarray, weights: np.ndarray):
        r = np.ascontiguousarray(rates, dtype=np.float64)
        w = np.ascontiguousarray(weights, dtype=np.float64)
        self._check(self._lib.phylo_set_categories(self._ctx, _dptr(r),
                                                   _dptr(w)))

    def set_branch_lengths(self, t):
        """t: numpy FP64 [2N-2] (host) or a CUDA FP64 tensor (device)."""
        if hasattr(t, "is_cuda") and t.is_cuda:
            import torch
            assert t.dtype == torch.float64 and t.numel() == 2 * self.n_tips - 2
            t = t.contiguous()
            self._t_keep = t
            self._check(self._lib.phylo_set_branch_lengths(
                self._ctx, ctypes.c_void_p(t.data_ptr()), 1))
        else:
            a = np.ascontiguousarray(t, dtype=np.float64)
            assert a.shape == (2 * self.n_tips - 2,)
            if hasattr(t, "data_ptr") and not isinstance(t, np.ndarray):
                ptr = t.data_ptr()  # pinned torch tensor on the host
                self._t_keep = t
            else:
                ptr = a.ctypes.data
                self._t_keep = a
            self._check(self._lib.phylo_set_branch_lengths(
                self._ctx, ctypes.c_void_p(ptr), 0))

    # -- evaluation ---------------------------------------------------------
    def evaluate(self, gradient=True):
        """log P(Y) and (optionally) the gradient as a numpy FP64 array."""
        logL = ctypes.c_double(0.0)
        g = np.zeros(2 * self.n_tips - 2) if gradient else None
        self._check(self._lib.phylo_evaluate(
            self._ctx, ctypes.byref(logL), _dptr(g) if g is not None else None))
        return (float(logL.value), g) if gradient else float(logL.value)

    def evaluate_into(self, logL_host, grad_host):
        """Evaluate into caller-provided host buffers (e.g. pinned tensors):
        logL_host is a 1-element FP64 buffer, grad_host has 2N-2 entries."""
        self._check(self._lib.phylo_evaluate(
            self._ctx, ctypes.cast(ctypes.c_void_p(logL_host.data_ptr()),
                                   ctypes.POINTER(ctypes.c_double)),
            ctypes.cast(ctypes.c_void_p(grad_host.data_ptr()),
                        ctypes.POINTER(ctypes.c_double))))

    def evaluate_device(self, out=None):
        """Asynchronous evaluation into a CUDA FP64 tensor [2N-1] =
        [log P(Y), gradient...] on the context's stream."""
        import torch
        if out is None:
            if self._out is None:
                self._out = torch.empty(2 * self.n_tips - 1,
                                        dtype=torch.float64,
                                        device=self.device)
            out = self._out
        self._check(self._lib.phylo_evaluate_device(
            self._ctx, ctypes.c_void_p(out.data_ptr())))
        return out

    def evaluate_device_timed(self, events, out=None):
        """evaluate_device with five torch.cuda.Event(enable_timing=True)
        recorded at the phase boundaries (matrices, post-order, pre-order +
        gradient, reduction)."""
        import torch
        if out is None:
            if self._out is None:
                self._out = torch.empty(2 * self.n_tips - 1,
                                        dtype=torch.float64,
                                        device=self.device)
            out = self._out
        for e in events:
            if not e.cuda_event:  # torch creates the CUDA event lazily
                e.record(torch.cuda.current_stream(self.device))
        arr = (ctypes.c_void_p * 5)(*[ctypes.c_void_p(e.cuda_event)
                                      for e in events])
        self._check(self._lib.phylo_evaluate_device_timed(
            self._ctx, ctypes.c_void_p(out.data_ptr()), arr))
        return out

    # -- chain-rule epilogues on the last evaluation's gradient ------------
    # Arguments are numpy arrays (host form, synchronous) or CUDA tensors
    # (device form, asynchronous on the context's stream; outputs are new
    # tensors on the same device).

    @staticmethod
    def _on_device(x):
        return not isinstance(x, np.ndarray) and getattr(x, "is_cuda", False)

    @staticmethod
    def _vptr(x):
        if isinstance(x, np.ndarray):
            return ctypes.c_void_p(x.ctypes.data)
        return ctypes.c_void_p(x.data_ptr())

    def _f64(self, x, n):
        if self._on_device(x):
            import torch
            t = x.to(torch.float64).contiguous()
            if t.numel() != n:
                raise ValueError(f"expected {n} values")
            return t
        a = np.ascontiguousarray(x, dtype=np.float64)
        if a.size != n:
            raise ValueError(f"expected {n} values")
        return a

    def _empty_like_input(self, ref, n):
        if self._on_device(ref):
            import torch
            return torch.empty(n, dtype=torch.float64, device=ref.device)
        return np.zeros(n)

    def gradient_rate_time(self, rates, times):
        """(d/d rates, d/d times) for t_i = rates_i times_i."""
        nb = 2 * self.n_tips - 2
        r, t = self._f64(rates, nb), self._f64(times, nb)
        dev = self._on_device(r)
        dr, dt = self._empty_like_input(r, nb), self._empty_like_input(r, nb)
        self._check(self._lib.phylo_gradient_rate_time(
            self._ctx, self._vptr(r), self._vptr(t), self._vptr(dr),
            self._vptr(dt), int(dev)))
        return dr, dt

    def gradient_heights(self, rates=None):
        """d/d h for t_i = rates_i (h_parent(i) - h_i); 2N-1 node heights."""
        nb, nn = 2 * self.n_tips - 2, 2 * self.n_tips - 1
        r = None if rates is None else self._f64(rates, nb)
        dev = r is not None and self._on_device(r)
        if r is None:
            out = np.zeros(nn)
        else:
            out = self._empty_like_input(r, nn)
        self._check(self._lib.phylo_gradient_heights(
            self._ctx, None if r is None else self._vptr(r), self._vptr(out),
            int(dev)))
        return out

    def gradient_branch_sum(self, branches, weights=None):
        """sum_j weights_j g_{branches_j} (a strict clock: weights = times)."""
        dev = self._on_device(branches)
        if dev:
            import torch
            b = branches.to(torch.int32).contiguous()
            n = b.numel()
            w = None if weights is None else self._f64(weights, n)
            out = torch.empty(1, dtype=torch.float64, device=b.device)
        else:
            b = np.ascontiguousarray(branches, dtype=np.int32)
            n = b.size
            w = None if weights is None else self._f64(weights, n)
            out = np.zeros(1)
        self._check(self._lib.phylo_gradient_branch_sum(
            self._ctx, self._vptr(b), None if w is None else self._vptr(w), n,
            self._vptr(out), int(dev)))
        return out if dev else float(out[0])

    def check(self):
        self._check(self._lib.phylo_check(self._ctx))

    def launches_per_evaluation(self) -> int:
        return int(self._lib.phylo_launches_per_evaluation(self._ctx))

    def level_counts(self):
        """(post-order launches, pre-order launches) of one evaluation."""
        a, b = ctypes.c_int(0), ctypes.c_int(0)
        self._check(self._lib.phylo_level_counts(self._ctx, ctypes.byref(a),
                                                 ctypes.byref(b)))
        return int(a.value), int(b.value)

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.phylo_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def from_workload(w, precision: Optional[str] = None, device=None,
                  stream=None, tip_partials=False,
                  use_graph=True) -> PhyloContext:
    """Context with every input of a synth.Workload set (branch lengths
    included)."""
    ctx = PhyloContext(w.n_tips, w.n_patterns, w.n_states, w.n_categories,
                       precision or w.precision, tip_partials=tip_partials,
                       device=device, stream=stream, use_graph=use_graph)
    ctx.set_tree(w.parent)
    ctx.set_tip_states(w.tip_states)
    ctx.set_pattern_weights(w.pattern_weights)
    ctx.set_rate_matrix(w.Q, w.pi)
    ctx.set_categories(w.rates, w.weights)
    ctx.set_branch_lengths(w.t)
    return ctx
