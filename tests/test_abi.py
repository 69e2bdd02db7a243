"""The C-ABI library loads and exports every symbol include/ttals.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2606_31061_b300 import ttals as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ttals.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ttals_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_31061_b300 import build
    build.build()
    return T.load()


def test_every_declared_symbol_is_exported(lib):
    decl = _declared()
    assert decl, "no declarations parsed"
    assert sorted(T.EXPORTS) == decl
    for name in decl:
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for code, name in T.STATUS.items():
        assert lib.ttals_status_string(code)
    assert lib.ttals_status_string(99) == b"unknown status"


def test_invalid_arguments_rejected_before_cuda(lib):
    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 2)(4, 0)
    ranks = (ctypes.c_int64 * 2)(2, 2)
    assert lib.ttals_create(2, dims, ranks, None, ctypes.byref(h)) == 1      # EINVAL: I_2 = 0
    dims = (ctypes.c_int64 * 1)(4)
    assert lib.ttals_create(1, dims, ranks, None, ctypes.byref(h)) == 1      # one slice mode
    cfg = T.Config(7, 1, 0, 0, 0, 0, 0, 0)
    dims = (ctypes.c_int64 * 2)(4, 4)
    assert lib.ttals_create(2, dims, ranks, ctypes.byref(cfg), ctypes.byref(h)) == 1   # bad dtype
    cfg = T.Config(0, 1, 0, 0, 0, 0, 0, 3)
    assert lib.ttals_create(2, dims, ranks, ctypes.byref(cfg), ctypes.byref(h)) == 1   # mode 3
    cfg = T.Config(2, 1, 0, 0, 0, 0, 2, 0)
    assert lib.ttals_create(2, dims, ranks, ctypes.byref(cfg), ctypes.byref(h)) == 1   # factor 2
    cfg = T.Config(2, 1, 0, 0, 5, 0, 0, 0)
    assert lib.ttals_create(2, dims, ranks, ctypes.byref(cfg), ctypes.byref(h)) == 1   # env_kernel 5
    cfg = T.Config(2, 1, 0, 0, 0, 3, 0, 0)
    assert lib.ttals_create(2, dims, ranks, ctypes.byref(cfg), ctypes.byref(h)) == 1   # k1_split 3
    cfg = T.Config(2, 1, 0, 0, 0, 0, 0, 0, 3, 0)
    assert lib.ttals_create(2, dims, ranks, ctypes.byref(cfg), ctypes.byref(h)) == 1   # solve_kernel 3
    cfg = T.Config(2, 1, 0, 0, 0, 0, 0, 0, 0, 6)
    assert lib.ttals_create(2, dims, ranks, ctypes.byref(cfg), ctypes.byref(h)) == 1   # factor_cluster 6
    ranks = (ctypes.c_int64 * 2)(65, 65)
    dims = (ctypes.c_int64 * 2)(100, 100)
    assert lib.ttals_create(2, dims, ranks, None, ctypes.byref(h)) == 1      # rank above 64
    assert lib.ttals_push_slice(None, None, 0, None) == 1
    assert lib.ttals_sync(None) == 1
    assert lib.ttals_device_bytes(None) == 0
    dims = (ctypes.c_int64 * 2)(64, 64)
    ranks = (ctypes.c_int64 * 2)(8, 8)
    assert lib.ttals_create_batch(0, 2, dims, ranks, None, ctypes.byref(h)) == 1      # no streams
    assert lib.ttals_create_batch(65, 2, dims, ranks, None, ctypes.byref(h)) == 1     # above TTALS_MAX_BATCH
    assert not h.value
    assert lib.ttals_push_batch(None, None, 0, None) == 1
    assert lib.ttals_push_batch_masked(None, None, 0, 1, None) == 1
    assert lib.ttals_batch_select(None, 0) == 1
    assert lib.ttals_batch_size(None) == 0


def test_no_device_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 2)(8, 8)
    ranks = (ctypes.c_int64 * 2)(2, 2)
    assert lib.ttals_create(2, dims, ranks, None, ctypes.byref(h)) == 3      # ECUDA, no fallback
    assert not h.value


class _FakeTensor:
    """Tensor metadata only (what the binding's argument checks read)."""

    def __init__(self, n=16, dtype="torch.float32", cuda=True, dev=0, contiguous=True):
        import types
        self.is_cuda, self._n, self.dtype, self._c = cuda, n, dtype, contiguous
        self.device = types.SimpleNamespace(index=dev if cuda else None)

    def numel(self):
        return self._n

    def is_contiguous(self):
        return self._c


def test_noalloc_wrapper_rejects_bad_arguments_on_the_host():
    """slice_error_noalloc validates what the C entry point cannot see (it gets one element
    count and raw pointers): each bad case raises EINVAL before any library call."""
    F = _FakeTensor
    good = dict(x=F(16, "torch.float16"), y=F(16, "torch.float32"), out2=F(2, "torch.float64"))
    T.check_noalloc_args(device=0, **good)          # control: accepted
    bad_cases = [
        dict(good, x=F(16, "torch.float16", cuda=False)),          # host tensor
        dict(good, y=F(15, "torch.float32")),                      # shorter y
        dict(good, y=F(17, "torch.float32")),                      # longer y
        dict(good, x=F(16, "torch.float16", contiguous=False)),    # strided x
        dict(good, y=F(16, "torch.float32", contiguous=False)),    # strided y
        dict(good, y=F(16, "torch.float16")),                      # y not float64/float32
        dict(good, x=F(16, "torch.int32")),                        # x not a float type
        dict(good, out2=F(2, "torch.float32")),                    # out2 not float64
        dict(good, out2=F(1, "torch.float64")),                    # out2 too small
        dict(good, out2=F(2, "torch.float64", dev=1)),             # out2 on another device
        dict(good, y=F(16, "torch.float32", dev=1)),               # y on another device
    ]
    for case in bad_cases:
        with pytest.raises(T.TTALSError) as ei:
            T.check_noalloc_args(device=0, **case)
        assert ei.value.code == 1
