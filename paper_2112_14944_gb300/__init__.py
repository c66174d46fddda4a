"""GB300 (sm_103a) implementation of the PPRviz hot path.

PPRviz (Zhang et al., "Effective and Efficient PageRank-based Positioning for
Graph Visualization", SIGMOD 2023): personalized PageRank for every node of a
view, degree-normalised DPPR and the PDist transform (Sec. 3.1, Eq. (1)), and
stress-majorization positioning over PDist (Sec. 5, Eq. (7); Appendix A.1).

All computation happens in the CUDA library libpprviz.so behind the C ABI in
include/pprviz.h. This package only marshals arguments: numpy arrays are host
buffers, torch CUDA tensors are device buffers. PyTorch is used for device
memory and streams.
"""
from __future__ import annotations

import weakref

import numpy as np

from . import _binding as B
from ._binding import (PPRVIZ_DEGREE_COUNT, PPRVIZ_DEVICE_PTRS, PPRVIZ_FP32, PPRVIZ_FP32_BF16TC, PPRVIZ_FP32_CSR,
                       PPRVIZ_FP32_TC, PPRVIZ_FP64, PPRVIZ_OUT_FP64, PPRVIZ_UNDIRECTED, PPRVIZ_VALIDATE, PPRVizError)

__all__ = ["Context", "Graph", "StressEnergy", "PPRVizError", "FP32", "FP32_CSR", "FP32_TC", "FP32_BF16TC", "FP64",
           "library_path"]

FP32 = PPRVIZ_FP32
FP32_CSR = PPRVIZ_FP32_CSR
FP32_TC = PPRVIZ_FP32_TC
FP32_BF16TC = PPRVIZ_FP32_BF16TC
FP64 = PPRVIZ_FP64


def library_path() -> str:
    return B.LIB_PATH


class Graph:
    """A graph uploaded to the device (opaque library handle)."""

    def __init__(self, ctx: "Context", handle: int, n: int):
        self.ctx = ctx
        self.h = handle
        self.n = n

    def degrees(self, out=None):
        """(d(v) as float64 numpy array or the given buffer, n, nnz, m)."""
        if out is None:
            out = np.empty(self.n, dtype=np.float64)
        n, nnz, m = B.pprviz_graph_degrees(self.ctx.h, self.h, out)
        return out, n, nnz, m

    def free(self):
        if self.h:
            B.pprviz_graph_free(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Context:
    """A library context on one CUDA device.

    With `torch_stream=True` the context runs on a dedicated torch CUDA stream
    that is ordered after the caller's current stream for every device-buffer
    call (and the current stream waits for it afterwards).
    """

    def __init__(self, device: int = 0, torch_stream: bool = False):
        self._stream = None
        handle = None
        if torch_stream:
            import torch
            self._stream = torch.cuda.Stream(device=device)
            handle = self._stream.cuda_stream
        self.device = device
        self._graphs = weakref.WeakSet()  # live graphs, freed by close()
        self.h = B.pprviz_create(device, handle)

    # -- stream ordering for device (torch) buffers --
    def _enter(self, dev):
        if dev and self._stream is not None:
            import torch
            self._stream.wait_stream(torch.cuda.current_stream(self.device))

    def _leave(self, dev, *tensors):
        if dev and self._stream is not None:
            import torch
            torch.cuda.current_stream(self.device).wait_stream(self._stream)
            for t in tensors:
                if t is not None and B._is_torch(t):
                    t.record_stream(self._stream)

    def close(self):
        if self.h:
            for g in list(self._graphs):
                g.free()
            B.pprviz_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_workspace_limit(self, nbytes: int):
        """Cap the context's device workspace (0 = no cap); calls that would
        exceed it fail with E_OOM."""
        B.pprviz_set_workspace_limit(self.h, nbytes)

    def stats(self) -> dict:
        return B.pprviz_get_stats(self.h)

    def sync(self):
        B.pprviz_sync(self.h)

    def profile(self, enable=True):
        """Reset the per-kernel-class counters; enable: False off, True every launch,
        N > 1 one in N launches of the hot classes (sweep, L^Y, apply, other)."""
        B.pprviz_profile(self.h, enable)

    def kernel_times(self) -> dict:
        """{class: (device ms of the timed launches, launches, timed launches)} since the last profile() call."""
        return B.pprviz_kernel_times(self.h)

    def upload(self, n, row_ptr, col, weights=None, validate=True, degree_count=False, directed=False) -> Graph:
        """Upload a CSR graph: undirected (both directions stored) unless
        `directed` (each row lists the node's out-neighbours)."""
        flags = ((0 if directed else PPRVIZ_UNDIRECTED) | (PPRVIZ_VALIDATE if validate else 0)
                 | (PPRVIZ_DEGREE_COUNT if degree_count else 0))
        dev = B._mem_flags(row_ptr, col, weights) == PPRVIZ_DEVICE_PTRS
        self._enter(dev)
        h = B.pprviz_graph_upload(self.h, n, row_ptr, col, weights, flags)
        self._leave(dev)
        gr = Graph(self, h, int(n))
        self._graphs.add(gr)
        return gr

    def upload_graph(self, g, validate=True) -> Graph:
        """Upload a synth.Graph-like object (n, row_ptr, col, weight[, directed])."""
        return self.upload(g.n, g.row_ptr, g.col, g.weight, validate=validate,
                           directed=bool(getattr(g, "directed", False)))

    def dppr(self, graph: Graph, view, alpha=0.15, eps=1e-6, precision=FP32, n_clamp=0, dppr_out=None,
             pdist_out=None, cert=True, out64=False):
        """DPPR and PDist of `view` (host numpy or device torch buffers).

        Output buffers may be given; else numpy arrays are allocated when the
        view is a numpy array. Returns (dppr, pdist, cert, status)."""
        k = len(view)
        dev = B._mem_flags(view, dppr_out, pdist_out) == PPRVIZ_DEVICE_PTRS
        if not dev:
            dt = np.float64 if out64 else np.float32
            if dppr_out is None:
                dppr_out = np.empty((k, k), dtype=dt)
            if pdist_out is None:
                pdist_out = np.empty((k, k), dtype=dt)
        mf = (PPRVIZ_DEVICE_PTRS if dev else 0) | (PPRVIZ_OUT_FP64 if out64 else 0)
        cert_out = np.empty(k, dtype=np.float64) if cert else None
        self._enter(dev)
        st = B.pprviz_dppr(self.h, graph.h, view, k, alpha, eps, precision, dppr_out, pdist_out, n_clamp,
                           cert_out, mf)
        self._leave(dev, view, dppr_out, pdist_out)
        return dppr_out, pdist_out, cert_out, st

    def level_dppr(self, graph: Graph, leaf_sets, alpha=0.15, eps=1e-6, n_clamp=0, out64=False):
        """Level-l DPPR and PDist between supernodes given by their leaf sets
        (a list of node-id arrays, disjoint and non-empty; Sec. 3.2, Eq. (2)).
        Returns (level DPPR, level PDist, certificates, status) as numpy arrays."""
        sizes = np.array([len(s) for s in leaf_sets], dtype=np.int64)
        leaf_ptr = np.zeros(len(leaf_sets) + 1, dtype=np.int64)
        np.cumsum(sizes, out=leaf_ptr[1:])
        leaf_idx = np.ascontiguousarray(np.concatenate([np.asarray(s, dtype=np.int32) for s in leaf_sets]))
        k = len(leaf_sets)
        dt = np.float64 if out64 else np.float32
        D = np.empty((k, k), dtype=dt)
        Pd = np.empty((k, k), dtype=dt)
        cert = np.empty(k, dtype=np.float64)
        st = B.pprviz_level_dppr(self.h, graph.h, k, leaf_ptr, leaf_idx, alpha, eps, D, Pd, n_clamp, cert,
                                 PPRVIZ_OUT_FP64 if out64 else 0)
        return D, Pd, cert, st

    def dpr(self, graph: Graph, alpha=0.15, eps=1e-12, out=None):
        """DPR index of every node (Sec. 4, Eq. (dnpr-dnppr); Sec. 4.3): the
        PageRank from d / m. `out`: a float64 device tensor to fill, else a
        numpy array is returned. Returns (dpr, L1 error bound)."""
        dev = out is not None and B._mem_flags(out) == PPRVIZ_DEVICE_PTRS
        if out is None:
            out = np.empty(graph.n, dtype=np.float64)
        self._enter(dev)
        cert = B.pprviz_dpr(self.h, graph.h, alpha, eps, out, PPRVIZ_DEVICE_PTRS if dev else 0)
        self._leave(dev, out)
        return out, cert

    def louvain_plus(self, graph: Graph, k, with_info=False):
        """Louvain+ supergraph hierarchy (Sec. 5; Appendix A): a list of
        parent arrays, levels 1..L, where entry A of level l is the level-l
        supernode of level-(l-1) node A (level 0 = the leaves). With
        with_info, also the call's counters (levels, rounds, visits)."""
        n = graph.n
        level_n = np.zeros(65, dtype=np.int64)
        cap = 2 * n + 64
        while True:
            parent = np.empty(cap, dtype=np.int32)
            ok, info = B.pprviz_louvain_plus(self.h, graph.h, k, level_n, 64, parent, cap)
            if ok:
                break
            if info["parent_need"] <= cap:
                raise RuntimeError("pprviz_louvain_plus: more than 64 levels")
            cap = info["parent_need"]  # a deep hierarchy: once more with room for it
        levels, off = [], 0
        for l in range(1, info["levels"] + 1):
            levels.append(parent[off:off + level_n[l - 1]].copy())
            off += level_n[l - 1]
        return (levels, info) if with_info else levels

    @staticmethod
    def leaf_csr(leaf_sets):
        """(leaf_ptr int64, leaf_idx int32) of a list of leaf-id arrays."""
        sizes = np.array([len(s) for s in leaf_sets], dtype=np.int64)
        leaf_ptr = np.zeros(len(leaf_sets) + 1, dtype=np.int64)
        np.cumsum(sizes, out=leaf_ptr[1:])
        leaf_idx = np.ascontiguousarray(np.concatenate([np.asarray(s, dtype=np.int32) for s in leaf_sets]))
        return leaf_ptr, leaf_idx

    def tau_push(self, graph: Graph, leaf_ptr, leaf_idx, dpr, alpha=0.15, eps=1 - 1 / np.e, delta=None, tau=0.0,
                 n_clamp=0, out64=True, ldppr_out=None, pdist_out=None, want_pdist=True):
        """Tau-Push (Sec. 4, Algorithms 1-3): (eps, delta)-approximate level-l
        DPPR between the children given by a leaf CSR, and its PDist.
        delta defaults to the paper's 1 / (10 k); tau <= 0 to 1 / sqrt(k n).
        Host (numpy) or device (torch) arrays, all of one kind; device calls
        write into ldppr_out / pdist_out. Returns (DPPR, PDist or None, info)."""
        k = len(leaf_ptr) - 1
        if delta is None:
            delta = 1.0 / (10 * k)
        dev = B._mem_flags(leaf_ptr, leaf_idx, dpr, ldppr_out, pdist_out) == PPRVIZ_DEVICE_PTRS
        dt = np.float64 if out64 else np.float32
        if not dev:
            ldppr_out = np.empty((k, k), dtype=dt) if ldppr_out is None else ldppr_out
            if want_pdist and pdist_out is None:
                pdist_out = np.empty((k, k), dtype=dt)
        mf = (PPRVIZ_DEVICE_PTRS if dev else 0) | (PPRVIZ_OUT_FP64 if out64 else 0)
        self._enter(dev)
        info = B.pprviz_tau_push(self.h, graph.h, k, leaf_ptr, leaf_idx, dpr, alpha, eps, delta, tau, ldppr_out,
                                 pdist_out if want_pdist else None, n_clamp, mf)
        self._leave(dev, ldppr_out, pdist_out)
        return ldppr_out, (pdist_out if want_pdist else None), info

    def frontier_profile(self, graph: Graph, view, sweeps, alpha=0.15, eps=1e-6):
        """Per power-iteration sweep, the (node, source) entries whose push
        residue is above GFP's threshold d(v) eps / max d (Algorithm 2)."""
        out = np.zeros(int(sweeps), dtype=np.int64)
        mf = B._mem_flags(view)
        B.pprviz_frontier_profile(self.h, graph.h, view, len(view), alpha, eps, sweeps, out, mf)
        return out

    def pdist(self, dppr, n_clamp, out=None):
        k = dppr.shape[0]
        dev = B._mem_flags(dppr, out) == PPRVIZ_DEVICE_PTRS
        f64 = (str(dppr.dtype).endswith("float64"))
        if out is None and not dev:
            out = np.empty((k, k), dtype=np.float64 if f64 else np.float32)
        mf = (PPRVIZ_DEVICE_PTRS if dev else 0) | (PPRVIZ_OUT_FP64 if f64 else 0)
        self._enter(dev)
        B.pprviz_pdist(self.h, dppr, k, n_clamp, out, mf)
        self._leave(dev, dppr, out)
        return out

    def layout(self, pdist, x0, iters, precision=FP32, x_out=None, stress=True):
        """Stress-majorization layout. Returns (X, final stress or None)."""
        k = pdist.shape[0]
        dev = B._mem_flags(pdist, x0, x_out) == PPRVIZ_DEVICE_PTRS
        f64 = str(pdist.dtype).endswith("float64")
        if x_out is None and not dev:
            x_out = np.empty((k, 2), dtype=np.float64 if f64 else np.float32)
        s = np.zeros(1, dtype=np.float64) if stress else None
        mf = (PPRVIZ_DEVICE_PTRS if dev else 0) | (PPRVIZ_OUT_FP64 if f64 else 0)
        self._enter(dev)
        B.pprviz_layout(self.h, pdist, k, x0, iters, precision, x_out, s, mf)
        self._leave(dev, pdist, x0, x_out)
        return x_out, (float(s[0]) if stress else None)

    def energy(self, pdist, x, grad_scale=1.0, grad_x=False, grad_pdist=False, gx_out=None, gd_out=None):
        """Stress energy (Eq. (7)) and optional gradients. Returns (E, grad_x, grad_pdist)."""
        k = pdist.shape[0]
        dev = B._mem_flags(pdist, x, gx_out, gd_out) == PPRVIZ_DEVICE_PTRS
        f64 = str(pdist.dtype).endswith("float64")
        if dev:
            import torch
            if grad_x and gx_out is None:
                gx_out = torch.empty((k, 2), dtype=pdist.dtype, device=pdist.device)
            if grad_pdist and gd_out is None:
                gd_out = torch.empty((k, k), dtype=pdist.dtype, device=pdist.device)
        else:
            dt = np.float64 if f64 else np.float32
            if grad_x and gx_out is None:
                gx_out = np.empty((k, 2), dtype=dt)
            if grad_pdist and gd_out is None:
                gd_out = np.empty((k, k), dtype=dt)
        e = np.zeros(1, dtype=np.float64)
        mf = (PPRVIZ_DEVICE_PTRS if dev else 0) | (PPRVIZ_OUT_FP64 if f64 else 0)
        self._enter(dev)
        B.pprviz_energy(self.h, pdist, k, x, grad_scale, e, gx_out if grad_x else None,
                        gd_out if grad_pdist else None, mf)
        self._leave(dev, pdist, x, gx_out, gd_out)
        return float(e[0]), (gx_out if grad_x else None), (gd_out if grad_pdist else None)

    def layout_metrics(self, x, graph: Graph = None, view=None):
        """(ND, ULCV) of a layout (Sec. 2): ND over all pairs of rows of x;
        ULCV over the graph's edges among the view's nodes (None without a
        graph). x: numpy (host) or torch CUDA tensor, float32 or float64."""
        k = x.shape[0]
        dev = B._mem_flags(x, view) == PPRVIZ_DEVICE_PTRS
        f64 = str(x.dtype).endswith("float64")
        nd = np.zeros(1, dtype=np.float64)
        ul = np.zeros(1, dtype=np.float64) if graph is not None else None
        mf = (PPRVIZ_DEVICE_PTRS if dev else 0) | (PPRVIZ_OUT_FP64 if f64 else 0)
        self._enter(dev)
        B.pprviz_layout_metrics(self.h, x, k, graph.h if graph is not None else None, view, nd, ul, mf)
        self._leave(dev, x, view)
        return float(nd[0]), (float(ul[0]) if ul is not None else None)

    def views_batch(self, graphs, x0_packed, alpha=0.15, eps=1e-6, iters=200, want_pdist=False, want_cert=False):
        """Batched views. x0_packed is a numpy array (host buffers) or a torch
        CUDA tensor (device buffers: the packed layouts and PDists come back as
        CUDA tensors). Returns (x_packed, pdist_packed, stress, offsets), plus
        the packed per-source certificates when want_cert is set."""
        sizes = np.array([g.n for g in graphs], dtype=np.int64)
        offsets = np.zeros(len(graphs) + 1, dtype=np.int64)
        np.cumsum(sizes, out=offsets[1:])
        nsq = int((sizes ** 2).sum())
        dev = B._is_torch(x0_packed)
        if dev:
            import torch
            x_packed = torch.empty_like(x0_packed)
            pd = torch.empty(nsq, dtype=torch.float32, device=x0_packed.device) if want_pdist else None
        else:
            x_packed = np.empty_like(x0_packed)
            pd = np.empty(nsq, dtype=np.float32) if want_pdist else None
        stress = np.zeros(len(graphs), dtype=np.float64)
        cert = np.full(int(offsets[-1]), np.nan, dtype=np.float64) if want_cert else None
        self._enter(dev)
        B.pprviz_views_batch(self.h, [g.h for g in graphs], offsets, alpha, eps, iters, x0_packed, pd, x_packed,
                             stress, cert, B.PPRVIZ_DEVICE_PTRS if dev else 0)
        self._leave(dev, x0_packed, pd, x_packed)
        if want_cert:
            return x_packed, pd, stress, offsets, cert
        return x_packed, pd, stress, offsets


def _make_stress_energy():
    import torch

    class StressEnergy(torch.autograd.Function):
        """L(X | Delta) of Eq. (7) with a hand-written backward.

        forward runs the library's energy kernel; backward re-runs it with the
        upstream gradient as `grad_scale`, recomputing every pair (no stored
        k x k intermediates). Inputs are CUDA tensors (float32 or float64)."""

        @staticmethod
        def forward(fctx, X, Delta, lib_ctx):
            e, _, _ = lib_ctx.energy(Delta.contiguous(), X.contiguous())
            fctx.save_for_backward(X, Delta)
            fctx.lib_ctx = lib_ctx
            return torch.tensor(e, dtype=X.dtype, device=X.device)

        @staticmethod
        def backward(fctx, grad_e):
            X, Delta = fctx.saved_tensors
            scale = float(grad_e)
            _, gx, gd = fctx.lib_ctx.energy(Delta.contiguous(), X.contiguous(), grad_scale=scale,
                                            grad_x=fctx.needs_input_grad[0], grad_pdist=fctx.needs_input_grad[1])
            return gx, gd, None

    return StressEnergy


class _Lazy:
    _cls = None

    def __get__(self, obj, owner):
        if _Lazy._cls is None:
            _Lazy._cls = _make_stress_energy()
        return _Lazy._cls


class _Namespace:
    StressEnergy = _Lazy()


def __getattr__(name):
    if name == "StressEnergy":
        return _Namespace.StressEnergy
    raise AttributeError(name)
