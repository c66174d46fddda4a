"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, and
exports every entry point that include/pprviz.h declares; the binding covers
each of them; calls that fail before touching a device return status codes."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pprviz.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pprviz_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2112_14944_gb300 import _binding as B
    if not os.path.exists(B.LIB_PATH):
        from paper_2112_14944_gb300 import build
        build.build()
    return B.load()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["pprviz_create", "pprviz_destroy", "pprviz_graph_upload", "pprviz_graph_free", "pprviz_dppr",
                 "pprviz_pdist", "pprviz_layout", "pprviz_energy", "pprviz_views_batch", "pprviz_sync",
                 "pprviz_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_wraps_every_declared_symbol(lib):
    from paper_2112_14944_gb300 import _binding as B
    assert set(_declared()) == set(B._SIGS)
    for name in _declared():
        assert callable(getattr(B, name)), name


def test_null_context_and_null_out_are_rejected(lib):
    from paper_2112_14944_gb300 import _binding as B
    assert lib.pprviz_sync(None) == B.PPRVIZ_E_INVALID_ARG
    assert lib.pprviz_get_stats(None, None) == B.PPRVIZ_E_INVALID_ARG
    assert lib.pprviz_create(None, 0, None) == B.PPRVIZ_E_INVALID_ARG
    assert lib.pprviz_dppr(None, None, None, 0, 0.15, 1e-6, 1, None, None, 0, None, 0) == B.PPRVIZ_E_INVALID_ARG
    assert lib.pprviz_last_error(None) == b"null context"


def test_create_on_a_missing_device_is_an_error_not_a_crash(lib):
    from paper_2112_14944_gb300 import _binding as B
    h = ctypes.c_void_p()
    st = lib.pprviz_create(ctypes.byref(h), 10_000, None)
    assert st == B.PPRVIZ_E_INVALID_ARG and not h.value


def test_binding_rejects_mixed_memory_spaces():
    torch = pytest.importorskip("torch")
    from paper_2112_14944_gb300 import _binding as B
    a = np.zeros(4, dtype=np.int32)
    assert B._mem_flags(a, None) == 0
    t = torch.zeros(4)
    assert B._mem_flags(t) == 0  # a CPU tensor is a host buffer
    with pytest.raises(ValueError):
        B._ptr(np.zeros((4, 4))[:, :2])  # non-contiguous


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2112_14944_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f


def test_noalloc_binding_rejects_bad_buffers_before_the_call():
    """The allocation-free entry point has no context to check buffers
    against, so its binding rejects wrong types, short buffers and host
    buffers before any C call (the C call is never reached here)."""
    torch = pytest.importorskip("torch")
    from paper_2112_14944_gb300 import _binding as B
    k = 8
    ok_d, ok_x = torch.zeros(k * k), torch.zeros(k * 2)
    with pytest.raises(ValueError, match="float32"):
        B._check_noalloc_buffers(k, torch.zeros(k * k, dtype=torch.float64), ok_x, None, None)
    with pytest.raises(ValueError, match="float32"):
        B._check_noalloc_buffers(k, ok_d, ok_x, torch.zeros(k * 2, dtype=torch.float16), None)
    with pytest.raises(ValueError, match="needs 64"):
        B._check_noalloc_buffers(k, torch.zeros(k * k - 1), ok_x, None, None)
    with pytest.raises(ValueError, match="needs 16"):
        B._check_noalloc_buffers(k, ok_d, torch.zeros(15), None, None)
    with pytest.raises(ValueError, match="needs 16"):
        B._check_noalloc_buffers(k, ok_d, ok_x, torch.zeros(3), None)
    with pytest.raises(ValueError, match="needs 64"):
        B._check_noalloc_buffers(k, ok_d, ok_x, None, torch.zeros(10))
    with pytest.raises(ValueError, match="device buffer"):
        B._check_noalloc_buffers(k, ok_d, ok_x, None, None)       # host tensors
    with pytest.raises(ValueError, match="torch CUDA tensor"):
        B._check_noalloc_buffers(k, np.zeros(k * k, np.float32), ok_x, None, None)
    with pytest.raises(ValueError, match="needs pdist and x"):
        B._check_noalloc_buffers(k, None, ok_x, None, None)
