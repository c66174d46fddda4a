"""ctypes binding of libpprviz (include/pprviz.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy arrays
(host buffers) and torch CUDA tensors (device buffers, PPRVIZ_DEVICE_PTRS) to
pointers and raises on a non-zero status. Loading fails loudly when the
compiled library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpprviz.so")

PPRVIZ_OK = 0
PPRVIZ_E_INVALID_ARG = 1
PPRVIZ_E_BAD_GRAPH = 2
PPRVIZ_E_OOM = 3
PPRVIZ_E_CUDA = 4
PPRVIZ_E_NOT_CONVERGED = 5
PPRVIZ_E_TIMEOUT = 6
PPRVIZ_UNDIRECTED = 1
PPRVIZ_VALIDATE = 2
PPRVIZ_DEGREE_COUNT = 4
PPRVIZ_DEVICE_PTRS = 1
PPRVIZ_OUT_FP64 = 2
PPRVIZ_FP64 = 0
PPRVIZ_FP32 = 1
PPRVIZ_FP32_CSR = 2
PPRVIZ_FP32_TC = 3
PPRVIZ_FP32_BF16TC = 4
KERNEL_CLASSES = ["graph", "sweep", "residual", "extract", "pdist", "factor", "ly", "apply", "energy", "other",
                  "push", "hier"]

STATUS_NAMES = {0: "OK", 1: "E_INVALID_ARG", 2: "E_BAD_GRAPH", 3: "E_OOM", 4: "E_CUDA",
                5: "E_NOT_CONVERGED", 6: "E_TIMEOUT"}

# Every entry point declared in include/pprviz.h, with its ctypes signature.
_VP = C.c_void_p
_SIGS = {
    "pprviz_create": (C.c_int, [C.POINTER(_VP), C.c_int, _VP]),
    "pprviz_destroy": (None, [_VP]),
    "pprviz_set_workspace_limit": (C.c_int, [_VP, C.c_int64]),
    "pprviz_test_expire_wait": (C.c_int, [_VP]),
    "pprviz_last_error": (C.c_char_p, [_VP]),
    "pprviz_sync": (C.c_int, [_VP]),
    "pprviz_get_stats": (C.c_int, [_VP, _VP]),
    "pprviz_profile": (C.c_int, [_VP, C.c_int]),
    "pprviz_kernel_times": (C.c_int, [_VP, _VP, _VP, _VP]),
    "pprviz_graph_upload": (C.c_int, [_VP, C.c_int64, _VP, _VP, _VP, C.c_uint32, C.c_uint32, C.POINTER(_VP)]),
    "pprviz_graph_free": (None, [_VP]),
    "pprviz_graph_degrees": (C.c_int, [_VP, _VP, _VP, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                       C.POINTER(C.c_double), C.c_uint32]),
    "pprviz_dppr": (C.c_int, [_VP, _VP, _VP, C.c_int32, C.c_double, C.c_double, C.c_int, _VP, _VP, C.c_int64,
                              _VP, C.c_uint32]),
    "pprviz_pdist": (C.c_int, [_VP, _VP, C.c_int32, C.c_int64, _VP, C.c_uint32]),
    "pprviz_frontier_profile": (C.c_int, [_VP, _VP, _VP, C.c_int32, C.c_double, C.c_double, C.c_int32, _VP,
                                          C.c_uint32]),
    "pprviz_level_dppr": (C.c_int, [_VP, _VP, C.c_int32, _VP, _VP, C.c_double, C.c_double, _VP, _VP, C.c_int64, _VP,
                                    C.c_uint32]),
    "pprviz_layout": (C.c_int, [_VP, _VP, C.c_int32, _VP, C.c_int32, C.c_int, _VP, _VP, C.c_uint32]),
    "pprviz_energy": (C.c_int, [_VP, _VP, C.c_int32, _VP, C.c_double, _VP, _VP, _VP, C.c_uint32]),
    "pprviz_views_batch": (C.c_int, [_VP, C.c_int32, _VP, _VP, C.c_double, C.c_double, C.c_int32, _VP, _VP, _VP,
                                     _VP, _VP, C.c_uint32]),
    "pprviz_energy_noalloc": (C.c_int, [_VP, C.c_int32, _VP, C.c_double, _VP, _VP, _VP, _VP]),
    "pprviz_layout_metrics": (C.c_int, [_VP, _VP, C.c_int32, _VP, _VP, _VP, _VP, C.c_uint32]),
    "pprviz_dpr": (C.c_int, [_VP, _VP, C.c_double, C.c_double, _VP, _VP, C.c_uint32]),
    "pprviz_louvain_plus": (C.c_int, [_VP, _VP, C.c_int32, _VP, C.c_int32, _VP, C.c_int64, _VP]),
    "pprviz_tau_push": (C.c_int, [_VP, _VP, C.c_int32, _VP, _VP, _VP, C.c_double, C.c_double, C.c_double, C.c_double,
                                  _VP, _VP, C.c_int64, _VP, C.c_uint32]),
}


class pprviz_stats(C.Structure):
    _fields_ = [("groups", C.c_int32), ("sweeps_main", C.c_int32), ("sweeps_refine", C.c_int32),
                ("refine_passes", C.c_int32), ("residual_passes", C.c_int32), ("kernel_launches", C.c_int32),
                ("max_cert", C.c_double), ("layout_iters", C.c_int32), ("source_group", C.c_int32),
                ("bytes_sweep", C.c_double), ("bytes_ly", C.c_double), ("bytes_apply", C.c_double),
                ("flops_factor", C.c_double), ("flops_dense", C.c_double), ("graph_launched", C.c_int32)]


class pprviz_tau_info(C.Structure):
    _fields_ = [("tau", C.c_double), ("r_max", C.c_double), ("backward_targets", C.c_int32),
                ("fwd_rounds", C.c_int32), ("bwd_rounds", C.c_int32), ("pad0", C.c_int32),
                ("fwd_pushes", C.c_int64), ("bwd_pushes", C.c_int64), ("fwd_edges", C.c_int64),
                ("bwd_edges", C.c_int64)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libpprviz.so; raises RuntimeError if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libpprviz.so not found at {path}: build it with "
                           "`python -m paper_2112_14944_gb300.build` (no CPU fallback exists)")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class PPRVizError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(ctx_ptr, status, allow=()):
    if status != PPRVIZ_OK and status not in allow:
        msg = load().pprviz_last_error(ctx_ptr)
        raise PPRVizError(status, msg.decode() if msg else "")
    return status


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, is_device) of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None, None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), x.is_cuda
    if not isinstance(x, np.ndarray) or not x.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be a C-contiguous numpy array")
    return x.ctypes.data, False


def _mem_flags(*bufs):
    dev = None
    for b in bufs:
        _, d = _ptr(b)
        if d is None:
            continue
        if dev is None:
            dev = d
        elif dev != d:
            raise ValueError("mix of host and device buffers in one call")
    return PPRVIZ_DEVICE_PTRS if dev else 0


# ----------------------------------------------------------------------------
# thin functions, one per entry point, same names as the C ABI
# ----------------------------------------------------------------------------
def pprviz_create(device: int = 0, cuda_stream: int | None = None) -> int:
    h = _VP()
    st = load().pprviz_create(C.byref(h), device, cuda_stream)
    if st != PPRVIZ_OK:
        raise PPRVizError(st, "pprviz_create failed")
    return h.value


def pprviz_destroy(ctx: int) -> None:
    load().pprviz_destroy(ctx)


def pprviz_set_workspace_limit(ctx: int, nbytes: int) -> None:
    _check(ctx, load().pprviz_set_workspace_limit(ctx, int(nbytes)))


def pprviz_test_expire_wait(ctx: int) -> None:
    _check(ctx, load().pprviz_test_expire_wait(ctx))


def pprviz_last_error(ctx: int) -> str:
    m = load().pprviz_last_error(ctx)
    return m.decode() if m else ""


def pprviz_sync(ctx: int) -> None:
    _check(ctx, load().pprviz_sync(ctx))


def pprviz_get_stats(ctx: int) -> dict:
    s = pprviz_stats()
    _check(ctx, load().pprviz_get_stats(ctx, C.addressof(s)))
    return {name: getattr(s, name) for name, _ in s._fields_}


def pprviz_profile(ctx: int, enable) -> None:
    """enable: False/0 off, True/1 every launch, N > 1 one in N launches of the hot classes."""
    _check(ctx, load().pprviz_profile(ctx, int(enable)))


def pprviz_kernel_times(ctx: int) -> dict:
    """{class: (device ms of the timed launches, launches, timed launches)} since the last pprviz_profile."""
    ms = np.zeros(len(KERNEL_CLASSES), dtype=np.float64)
    cnt = np.zeros(len(KERNEL_CLASSES), dtype=np.int64)
    timed = np.zeros(len(KERNEL_CLASSES), dtype=np.int64)
    _check(ctx, load().pprviz_kernel_times(ctx, ms.ctypes.data, cnt.ctypes.data, timed.ctypes.data))
    return {name: (float(ms[i]), int(cnt[i]), int(timed[i])) for i, name in enumerate(KERNEL_CLASSES)}


def pprviz_graph_upload(ctx, n, row_ptr, col_idx, weights=None, flags=PPRVIZ_UNDIRECTED | PPRVIZ_VALIDATE) -> int:
    mf = _mem_flags(row_ptr, col_idx, weights)
    h = _VP()
    _check(ctx, load().pprviz_graph_upload(ctx, int(n), _ptr(row_ptr)[0], _ptr(col_idx)[0], _ptr(weights)[0],
                                           flags, mf, C.byref(h)))
    return h.value


def pprviz_graph_free(g: int) -> None:
    load().pprviz_graph_free(g)


def pprviz_graph_degrees(ctx, g, deg_out=None):
    n = C.c_int64()
    nnz = C.c_int64()
    m = C.c_double()
    mf = _mem_flags(deg_out)
    _check(ctx, load().pprviz_graph_degrees(ctx, g, _ptr(deg_out)[0], C.byref(n), C.byref(nnz), C.byref(m), mf))
    return n.value, nnz.value, m.value


def pprviz_dppr(ctx, g, view, k, alpha, eps, precision, dppr_out, pdist_out, n_clamp, cert_out, mem_flags):
    return _check(ctx, load().pprviz_dppr(ctx, g, _ptr(view)[0], int(k), float(alpha), float(eps), int(precision),
                                          _ptr(dppr_out)[0], _ptr(pdist_out)[0], int(n_clamp), _ptr(cert_out)[0],
                                          mem_flags), allow=(PPRVIZ_E_NOT_CONVERGED,))


def pprviz_level_dppr(ctx, g, nsup, leaf_ptr, leaf_idx, alpha, eps, ldppr_out, pdist_out, n_clamp, cert_out,
                      mem_flags):
    return _check(ctx, load().pprviz_level_dppr(ctx, g, int(nsup), _ptr(leaf_ptr)[0], _ptr(leaf_idx)[0], float(alpha),
                                                float(eps), _ptr(ldppr_out)[0], _ptr(pdist_out)[0], int(n_clamp),
                                                _ptr(cert_out)[0], mem_flags), allow=(PPRVIZ_E_NOT_CONVERGED,))


def pprviz_dpr(ctx, g, alpha, eps, dpr_out, mem_flags):
    """Returns the certificate (1 - alpha)^(T + 1)."""
    cert = C.c_double()
    _check(ctx, load().pprviz_dpr(ctx, g, float(alpha), float(eps), _ptr(dpr_out)[0], C.byref(cert), mem_flags))
    return cert.value


class pprviz_louvain_info(C.Structure):
    _fields_ = [("levels", C.c_int32), ("rounds", C.c_int32), ("parent_need", C.c_int64),
                ("slot_visits", C.c_int64), ("pair_visits", C.c_int64), ("list_visits", C.c_int64),
                ("node_visits", C.c_int64)]


def pprviz_louvain_plus(ctx, g, k, level_n, level_cap, parent, parent_cap):
    """level_n / parent: host numpy int64 / int32 arrays. Returns (ok, info
    dict); ok is False (and info holds levels and parent_need) when the
    outputs were too short, any other failure raises."""
    info = pprviz_louvain_info()
    st = load().pprviz_louvain_plus(ctx, g, int(k), _ptr(level_n)[0], int(level_cap), _ptr(parent)[0],
                                    int(parent_cap), C.byref(info))
    out = {name: getattr(info, name) for name, _ in info._fields_}
    if st == PPRVIZ_E_INVALID_ARG and info.parent_need > 0:  # written only once the hierarchy is built
        return False, out
    _check(ctx, st)
    return True, out


def pprviz_tau_push(ctx, g, nsup, leaf_ptr, leaf_idx, dpr, alpha, eps, delta, tau, ldppr_out, pdist_out, n_clamp,
                    mem_flags):
    """Returns the call's pprviz_tau_info as a dict."""
    info = pprviz_tau_info()
    _check(ctx, load().pprviz_tau_push(ctx, g, int(nsup), _ptr(leaf_ptr)[0], _ptr(leaf_idx)[0], _ptr(dpr)[0],
                                       float(alpha), float(eps), float(delta), float(tau), _ptr(ldppr_out)[0],
                                       _ptr(pdist_out)[0], int(n_clamp), C.byref(info), mem_flags))
    return {name: getattr(info, name) for name, _ in info._fields_ if name != "pad0"}


def pprviz_frontier_profile(ctx, g, view, k, alpha, eps, sweeps, active_out, mem_flags):
    return _check(ctx, load().pprviz_frontier_profile(ctx, g, _ptr(view)[0], int(k), float(alpha), float(eps),
                                                      int(sweeps), _ptr(active_out)[0], mem_flags))


def pprviz_pdist(ctx, dppr, k, n_clamp, pdist_out, mem_flags):
    return _check(ctx, load().pprviz_pdist(ctx, _ptr(dppr)[0], int(k), int(n_clamp), _ptr(pdist_out)[0], mem_flags))


def pprviz_layout(ctx, pdist, k, x0, iters, precision, x_out, stress_out, mem_flags):
    return _check(ctx, load().pprviz_layout(ctx, _ptr(pdist)[0], int(k), _ptr(x0)[0], int(iters), int(precision),
                                            _ptr(x_out)[0], _ptr(stress_out)[0], mem_flags))


def pprviz_energy(ctx, pdist, k, x, grad_scale, e_out, grad_x, grad_pdist, mem_flags):
    return _check(ctx, load().pprviz_energy(ctx, _ptr(pdist)[0], int(k), _ptr(x)[0], float(grad_scale),
                                            _ptr(e_out)[0], _ptr(grad_x)[0], _ptr(grad_pdist)[0], mem_flags))


def pprviz_layout_metrics(ctx, x, k, g, view, nd_out, ulcv_out, mem_flags):
    return _check(ctx, load().pprviz_layout_metrics(ctx, _ptr(x)[0], int(k), g, _ptr(view)[0], _ptr(nd_out)[0],
                                                    _ptr(ulcv_out)[0], mem_flags))


def pprviz_views_batch(ctx, graphs, offsets, alpha, eps, iters, x0_packed, pdist_packed, x_packed, stress_out,
                       cert_out, mem_flags):
    arr = (_VP * len(graphs))(*graphs)
    return _check(ctx, load().pprviz_views_batch(ctx, len(graphs), C.addressof(arr), _ptr(offsets)[0], float(alpha),
                                                 float(eps), int(iters), _ptr(x0_packed)[0], _ptr(pdist_packed)[0],
                                                 _ptr(x_packed)[0], _ptr(stress_out)[0], _ptr(cert_out)[0],
                                                 mem_flags),
                  allow=(PPRVIZ_E_NOT_CONVERGED,))


def _check_noalloc_buffers(k, pdist, x, grad_x, grad_pdist):
    """The C entry point has no context and sees only pointers, so the sizes,
    element type and device of its buffers are checked here: float32 torch
    tensors holding at least k*k (pdist, grad_pdist) or k*2 (x, grad_x)
    elements, all on the current CUDA device. k outside [1, 65536] is left to
    the library, which rejects it with PPRVIZ_E_INVALID_ARG."""
    if pdist is None or x is None:
        raise ValueError("pprviz_energy_noalloc needs pdist and x")
    k = int(k)
    need = {"pdist": (pdist, k * k), "x": (x, 2 * k), "grad_x": (grad_x, 2 * k), "grad_pdist": (grad_pdist, k * k)}
    given = [(name, b, n) for name, (b, n) in need.items() if b is not None]
    for name, b, _ in given:
        if not _is_torch(b):
            raise ValueError(f"pprviz_energy_noalloc: {name} must be a torch CUDA tensor")
        if str(b.dtype) != "torch.float32":
            raise ValueError(f"pprviz_energy_noalloc: {name} must be float32, got {b.dtype}")
        if not b.is_contiguous():
            raise ValueError(f"pprviz_energy_noalloc: {name} must be contiguous")
    for name, b, n in given:
        if 1 <= k <= 65536 and b.numel() < n:
            raise ValueError(f"pprviz_energy_noalloc: {name} holds {b.numel()} elements, needs {n}")
    for name, b, _ in given:
        if not b.is_cuda:
            raise ValueError(f"pprviz_energy_noalloc: {name} must be a device buffer")
        import torch
        if b.device.index != torch.cuda.current_device():
            raise ValueError(f"pprviz_energy_noalloc: {name} is on cuda:{b.device.index}, "
                             f"the current device is cuda:{torch.cuda.current_device()}")


def pprviz_energy_noalloc(pdist, k, x, grad_scale=1.0, grad_x=None, grad_pdist=None, cuda_stream=None):
    """Energy and gradients through the allocation-free entry point: float32
    device (torch CUDA) buffers on the current device only, no context.
    Returns (status, energy)."""
    _check_noalloc_buffers(k, pdist, x, grad_x, grad_pdist)
    e = C.c_double(0.0)
    st = load().pprviz_energy_noalloc(_ptr(pdist)[0], int(k), _ptr(x)[0], float(grad_scale), C.byref(e),
                                      _ptr(grad_x)[0], _ptr(grad_pdist)[0], cuda_stream)
    return st, e.value
