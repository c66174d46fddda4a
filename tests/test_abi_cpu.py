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


def test_louvain_plus_null_context_and_host_marshalling(lib, monkeypatch):
    """pprviz_louvain_plus rejects a NULL context without touching a device;
    the Python method splits the concatenated parent arrays per level and,
    when the first buffer is short, calls again with the size the library
    reported (the library call is replaced by a fake here: no GPU)."""
    import paper_2112_14944_gb300 as P
    from paper_2112_14944_gb300 import _binding as B
    ln = np.zeros(65, np.int64)
    par = np.zeros(4, np.int32)
    info = B.pprviz_louvain_info()
    assert lib.pprviz_louvain_plus(None, None, 5, ln.ctypes.data, 64, par.ctypes.data, 4, ctypes.byref(info)) == \
        B.PPRVIZ_E_INVALID_ARG
    # a three-level hierarchy of 5000 leaves: 5000 -> 3000 -> 40 -> 2
    levels = [np.arange(5000) % 3000, np.arange(3000) % 40, np.arange(40) % 2]
    need = sum(len(p) for p in levels)
    calls = []

    def fake(ctx, g, k, level_n, level_cap, parent, parent_cap):
        calls.append(parent_cap)
        out = {"levels": 3, "rounds": 9, "parent_need": need, "slot_visits": 0, "pair_visits": 0,
               "list_visits": 0, "node_visits": 0}
        if parent_cap < need:
            return False, out
        level_n[:4] = [5000, 3000, 40, 2]
        parent[:need] = np.concatenate(levels)
        return True, out

    monkeypatch.setattr(B, "pprviz_louvain_plus", fake)

    class FakeGraph:
        n, h = 1000, 1  # the graph's n sets the first guess (2 n + 64 entries), below `need`

    ctx = P.Context.__new__(P.Context)
    ctx.h = 1
    got, info = ctx.louvain_plus(FakeGraph(), 25, with_info=True)
    ctx.h = 0
    assert calls == [2 * 1000 + 64, need] and info["levels"] == 3
    assert len(got) == 3 and all(np.array_equal(a, b) for a, b in zip(got, levels))
