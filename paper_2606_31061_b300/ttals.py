"""Thin Python binding of the libttals C ABI (include/ttals.h).

Argument marshalling only: every step of the update runs in the library's CUDA
kernels.  PyTorch supplies device memory and CUDA streams.  There is no CPU
fallback: if the library or a CUDA device is missing, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libttals.so")

F64, F32, F16, BF16 = 0, 1, 2, 3
DTYPES = {"f64": F64, "f32": F32, "f16": F16, "bf16": BF16}
MODES = {"literal": 0, "lsq": 1, "noortho": 2}   # ttals_config.mode
MAX_BATCH = 64          # TTALS_MAX_BATCH: streams per ttals_create_batch
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENONFINITE", 5: "ETIMEOUT", 6: "ESTATE"}

# every symbol include/ttals.h declares (checked by the ABI test)
EXPORTS = ("ttals_create", "ttals_destroy", "ttals_effective_ranks", "ttals_set_cores",
           "ttals_push_slice", "ttals_reconstruct", "ttals_cores", "ttals_stats", "ttals_step",
           "ttals_sync", "ttals_device_bytes", "ttals_status_string", "ttals_last_error",
           "ttals_launch_count", "ttals_stats_async", "ttals_profile", "ttals_profile_read",
           "ttals_slice_error_noalloc", "ttals_create_batch", "ttals_push_batch", "ttals_batch_select",
           "ttals_batch_size", "ttals_push_batch_masked", "ttals_widen_u8", "ttals_seed_cores",
           "ttals_debug_stall_solve", "ttals_batch_ingest_init", "ttals_batch_push_host",
           "ttals_batch_ticket_done")


class TTALSError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str = ""):
        self.code = code
        self.name = STATUS.get(code, str(code))
        super().__init__(f"{where}: {self.name}" + (f" ({msg})" if msg else ""))


class Config(ctypes.Structure):
    _fields_ = [("ingest", ctypes.c_int), ("seed", ctypes.c_uint64), ("device", ctypes.c_int),
                ("qr_passes", ctypes.c_int), ("env_kernel", ctypes.c_int), ("k1_split", ctypes.c_int),
                ("factor", ctypes.c_int), ("mode", ctypes.c_int), ("solve_kernel", ctypes.c_int),
                ("factor_cluster", ctypes.c_int)]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libttals.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} is missing; build it with python -m paper_2606_31061_b300.build")
    lib = ctypes.CDLL(path)
    P, I64P, VP = ctypes.POINTER, ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p
    sig = {
        "ttals_create": (ctypes.c_int, [ctypes.c_int, I64P, I64P, P(Config), P(VP)]),
        "ttals_destroy": (None, [VP]),
        "ttals_effective_ranks": (ctypes.c_int, [VP, I64P]),
        "ttals_set_cores": (ctypes.c_int, [VP, P(P(ctypes.c_double)), P(ctypes.c_double), ctypes.c_int64]),
        "ttals_push_slice": (ctypes.c_int, [VP, VP, ctypes.c_int, VP]),
        "ttals_reconstruct": (ctypes.c_int, [VP, VP, ctypes.c_int, VP]),
        "ttals_cores": (ctypes.c_int, [VP, ctypes.c_int, P(ctypes.c_double), ctypes.c_size_t]),
        "ttals_stats": (ctypes.c_int, [VP, P(ctypes.c_double)]),
        "ttals_step": (ctypes.c_int, [VP, I64P]),
        "ttals_sync": (ctypes.c_int, [VP]),
        "ttals_device_bytes": (ctypes.c_size_t, [VP]),
        "ttals_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "ttals_last_error": (ctypes.c_char_p, []),
        "ttals_launch_count": (ctypes.c_uint64, [VP]),
        "ttals_stats_async": (ctypes.c_int, [VP, VP, VP]),
        "ttals_profile": (ctypes.c_int, [VP, ctypes.c_int]),
        "ttals_profile_read": (ctypes.c_int, [VP, P(ctypes.c_double), I64P]),
        "ttals_slice_error_noalloc": (ctypes.c_int, [VP, ctypes.c_int, VP, ctypes.c_int, ctypes.c_int64, VP, VP]),
        "ttals_create_batch": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, I64P, I64P, P(Config), P(VP)]),
        "ttals_push_batch": (ctypes.c_int, [VP, VP, ctypes.c_int, VP]),
        "ttals_batch_select": (ctypes.c_int, [VP, ctypes.c_int]),
        "ttals_push_batch_masked": (ctypes.c_int, [VP, VP, ctypes.c_int, ctypes.c_uint64, VP]),
        "ttals_widen_u8": (ctypes.c_int, [VP, VP, ctypes.c_int, ctypes.c_int64, VP]),
        "ttals_batch_size": (ctypes.c_int, [VP]),
        "ttals_seed_cores": (ctypes.c_int, [VP, ctypes.c_uint64]),
        "ttals_debug_stall_solve": (ctypes.c_int, [VP, ctypes.c_int]),
        "ttals_batch_ingest_init": (ctypes.c_int, [VP, ctypes.c_int]),
        "ttals_batch_push_host": (ctypes.c_int, [VP, ctypes.c_int, P(ctypes.c_int), P(VP), P(ctypes.c_uint64)]),
        "ttals_batch_ticket_done": (ctypes.c_int, [VP, ctypes.c_uint64, P(ctypes.c_int)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(code: int, where: str):
    if code != 0:
        msg = load().ttals_last_error().decode() if code == 3 else ""
        raise TTALSError(code, where, msg)


def _i64(seq):
    return (ctypes.c_int64 * len(seq))(*[int(v) for v in seq])


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Stream:
    """One Online TT-ALS stream (a ttals_stream handle), or with n_streams > 0 a batch of that
    many streams of one shape (ttals_create_batch) that step together (push_batch); the
    per-stream methods then refer to the stream chosen by select()."""

    def __init__(self, dims: Sequence[int], ranks: Sequence[int], ingest: str = "f64",
                 seed: int = 0x5EED, device: int = 0, qr_passes: int = 0, n_streams: int = 0,
                 env_kernel: int = 0, k1_split: int = 0, factor: str = "fp64", mode: str = "literal",
                 solve_kernel: int = 0, factor_cluster: int = 0):
        lib = load()
        self.dims = tuple(int(d) for d in dims)
        self.ingest = ingest
        if factor not in ("fp64", "fp32"):
            raise ValueError(f"factor must be 'fp64' or 'fp32', not {factor!r}")
        if mode not in MODES:
            raise ValueError(f"mode must be one of {sorted(MODES)}, not {mode!r}")
        cfg = Config(DTYPES[ingest], seed, device, qr_passes, env_kernel, k1_split, 0 if factor == "fp64" else 1,
                     MODES[mode], solve_kernel, factor_cluster)
        h = ctypes.c_void_p()
        if n_streams > 0:
            code = lib.ttals_create_batch(int(n_streams), len(self.dims), _i64(self.dims), _i64(ranks),
                                          ctypes.byref(cfg), ctypes.byref(h))
            if code != 0:
                raise TTALSError(code, "ttals_create_batch", lib.ttals_last_error().decode())
        else:
            _check(lib.ttals_create(len(self.dims), _i64(self.dims), _i64(ranks), ctypes.byref(cfg),
                                    ctypes.byref(h)), "ttals_create")
        self._h = h
        self.n_streams = int(lib.ttals_batch_size(h))
        out = (ctypes.c_int64 * len(self.dims))()
        _check(lib.ttals_effective_ranks(h, out), "ttals_effective_ranks")
        self.ranks = tuple(int(v) for v in out)
        self.full = (1,) + self.ranks

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            load().ttals_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls
    def set_cores(self, cores, g, t: int = 0):
        arrs = [np.ascontiguousarray(c, dtype=np.float64) for c in cores]
        for k, a in enumerate(arrs):
            want = (self.full[k], self.dims[k], self.full[k + 1])
            if a.shape != want:
                raise ValueError(f"core {k + 1} shape {a.shape} != {want}")
        gg = np.ascontiguousarray(g, dtype=np.float64).reshape(-1)
        ptrs = (ctypes.POINTER(ctypes.c_double) * len(arrs))(
            *[a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for a in arrs])
        _check(load().ttals_set_cores(self._h, ptrs, gg.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      int(t)), "ttals_set_cores")

    def seed_cores(self, seed: int):
        """ttals_seed_cores: the library's default random initial cores drawn from `seed`
        (those ttals_create gives for cfg.seed = seed), t = 0."""
        _check(load().ttals_seed_cores(self._h, ctypes.c_uint64(int(seed))), "ttals_seed_cores")

    def push(self, slice_tensor, stream=None):
        """Enqueue one update for a contiguous device tensor of the ingest dtype."""
        _check(load().ttals_push_slice(self._h, ctypes.c_void_p(slice_tensor.data_ptr()),
                                       DTYPES[self.ingest], ctypes.c_void_p(_stream_handle(stream))),
               "ttals_push_slice")

    def push_ptr(self, ptr: int, stream_handle: int):
        _check(load().ttals_push_slice(self._h, ctypes.c_void_p(ptr), DTYPES[self.ingest],
                                       ctypes.c_void_p(stream_handle)), "ttals_push_slice")

    def reconstruct(self, out_tensor, dtype: str = "f64", stream=None):
        _check(load().ttals_reconstruct(self._h, ctypes.c_void_p(out_tensor.data_ptr()), DTYPES[dtype],
                                        ctypes.c_void_p(_stream_handle(stream))), "ttals_reconstruct")

    def core(self, k: int) -> np.ndarray:
        m = len(self.dims)
        shape = (self.full[k - 1], self.dims[k - 1], self.full[k]) if k <= m else (self.full[m],)
        out = np.empty(shape, dtype=np.float64)
        _check(load().ttals_cores(self._h, k, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  out.size), "ttals_cores")
        return out

    def cores(self):
        m = len(self.dims)
        return [self.core(k) for k in range(1, m + 1)], self.core(m + 1)

    def stats(self) -> np.ndarray:
        out = (ctypes.c_double * 4)()
        _check(load().ttals_stats(self._h, out), "ttals_stats")
        return np.array(list(out))

    def step(self) -> int:
        t = ctypes.c_int64()
        _check(load().ttals_step(self._h, ctypes.byref(t)), "ttals_step")
        return t.value

    def sync(self):
        _check(load().ttals_sync(self._h), "ttals_sync")

    def sync_status(self) -> int:
        """ttals_sync's status code without raising."""
        return load().ttals_sync(self._h)

    @property
    def device_bytes(self) -> int:
        return int(load().ttals_device_bytes(self._h))

    @property
    def launch_count(self) -> int:
        return int(load().ttals_launch_count(self._h))

    def stats_async(self, out_ptr: int, stream=None):
        _check(load().ttals_stats_async(self._h, ctypes.c_void_p(out_ptr),
                                        ctypes.c_void_p(_stream_handle(stream))), "ttals_stats_async")

    def push_batch(self, slices, stream=None, active: Optional[int] = None):
        """ttals_push_batch: one step of every stream; `slices` is a contiguous CUDA tensor of
        n_streams slices (stream b's slice is slices[b]).  With `active` (bit b: stream b),
        only those streams step (ttals_push_batch_masked)."""
        self.push_batch_ptr(slices.data_ptr(), _stream_handle(stream), active)

    def push_batch_ptr(self, ptr: int, stream_handle: int, active: Optional[int] = None):
        """ttals_push_batch, or ttals_push_batch_masked when `active` (bit b: stream b) is given."""
        if active is None:
            _check(load().ttals_push_batch(self._h, ctypes.c_void_p(ptr), DTYPES[self.ingest],
                                           ctypes.c_void_p(stream_handle)), "ttals_push_batch")
        else:
            _check(load().ttals_push_batch_masked(self._h, ctypes.c_void_p(ptr), DTYPES[self.ingest],
                                                  ctypes.c_uint64(active), ctypes.c_void_p(stream_handle)),
                   "ttals_push_batch_masked")

    def ingest_init(self, u8: bool = False):
        """ttals_batch_ingest_init: the batch gets its own input blocks, copy/compute streams and
        completion events (u8: frames are 8-bit pixels widened on the device)."""
        _check(load().ttals_batch_ingest_init(self._h, 1 if u8 else 0), "ttals_batch_ingest_init")

    def push_host(self, slots: Sequence[int], host_ptrs: Sequence[int]) -> int:
        """ttals_batch_push_host: one masked step of the streams in `slots`, frame i copied from
        pinned host address host_ptrs[i]; returns the step's ticket."""
        n = len(slots)
        sl = (ctypes.c_int * n)(*[int(v) for v in slots])
        pp = (ctypes.c_void_p * n)(*[int(v) for v in host_ptrs])
        t = ctypes.c_uint64()
        _check(load().ttals_batch_push_host(self._h, n, sl, pp, ctypes.byref(t)), "ttals_batch_push_host")
        return t.value

    def ticket_done(self, ticket: int) -> bool:
        d = ctypes.c_int()
        _check(load().ttals_batch_ticket_done(self._h, ctypes.c_uint64(int(ticket)), ctypes.byref(d)),
               "ttals_batch_ticket_done")
        return bool(d.value)

    def select(self, index: int):
        """ttals_batch_select: later per-stream calls refer to stream `index` of the batch."""
        _check(load().ttals_batch_select(self._h, int(index)), "ttals_batch_select")

    def debug_stall_solve(self, n_pushes: int):
        """ttals_debug_stall_solve: the next n_pushes pushes time out in the local solve
        (bounded wait; ETIMEOUT latched, the step not committed).  Test hook."""
        _check(load().ttals_debug_stall_solve(self._h, int(n_pushes)), "ttals_debug_stall_solve")

    def profile(self, enable: bool):
        _check(load().ttals_profile(self._h, 1 if enable else 0), "ttals_profile")

    def profile_read(self):
        """(ms level-1 solve, ms level-1 factorisation, ms level-1 environment, ms whole update,
        pushes) summed since the last read."""
        ms = (ctypes.c_double * 4)()
        n = ctypes.c_int64()
        _check(load().ttals_profile_read(self._h, ms, ctypes.byref(n)), "ttals_profile_read")
        return ms[0], ms[1], ms[2], ms[3], n.value


def widen_u8(src, dst, stream=None):
    """ttals_widen_u8: dst (CUDA float16/bfloat16/float32/float64) = src (CUDA uint8), exact."""
    dt = DTYPES[_TORCH_DTYPES[str(dst.dtype).replace("torch.", "")]]
    _check(load().ttals_widen_u8(ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()), dt,
                                 ctypes.c_int64(src.numel()), ctypes.c_void_p(_stream_handle(stream))),
           "ttals_widen_u8")


_TORCH_DTYPES = {"float64": "f64", "float32": "f32", "float16": "f16", "bfloat16": "bf16"}


def check_noalloc_args(x, y, out2, device: int):
    """Argument checks of slice_error_noalloc, on tensor metadata only (no device access).

    The C entry point receives raw pointers and one element count and cannot see a short
    or strided y, an out2 that is too small, or a tensor on another device; any of those
    would make its kernel read or write out of bounds.  Raises TTALSError(EINVAL)."""
    def bad(why):
        raise TTALSError(1, "ttals_slice_error_noalloc", why)
    for name, t in (("x", x), ("y", y), ("out2", out2)):
        if not getattr(t, "is_cuda", False):
            bad(f"{name} is not a CUDA tensor")
        if t.device.index != device:
            bad(f"{name} is on cuda:{t.device.index}, the current device is cuda:{device}")
        if not t.is_contiguous():
            bad(f"{name} is not contiguous")
    if y.numel() != x.numel():
        bad(f"y has {y.numel()} elements, x has {x.numel()}")
    if str(x.dtype).replace("torch.", "") not in _TORCH_DTYPES:
        bad(f"x dtype {x.dtype} is not float64/float32/float16/bfloat16")
    if str(y.dtype).replace("torch.", "") not in ("float64", "float32"):
        bad(f"y dtype {y.dtype} is not float64/float32")
    if str(out2.dtype).replace("torch.", "") != "float64" or out2.numel() < 2:
        bad("out2 must be a float64 tensor of at least 2 elements")


def slice_error_noalloc(x, y, out2, stream=None):
    """ttals_slice_error_noalloc: enqueue out2[0] = ||x||^2, out2[1] = ||x - y||^2.

    x, y: contiguous CUDA tensors of the same element count on the current device
    (y float64 or float32); out2: a CUDA float64 tensor of at least 2 elements on the same
    device.  Allocates no device memory.  Bad arguments raise TTALSError(EINVAL) before the
    call (check_noalloc_args).
    """
    import torch
    check_noalloc_args(x, y, out2, torch.cuda.current_device())
    xt = DTYPES[_TORCH_DTYPES[str(x.dtype).replace("torch.", "")]]
    yt = DTYPES[_TORCH_DTYPES[str(y.dtype).replace("torch.", "")]]
    lib = load()
    code = lib.ttals_slice_error_noalloc(ctypes.c_void_p(x.data_ptr()), xt, ctypes.c_void_p(y.data_ptr()), yt,
                                         ctypes.c_int64(x.numel()), ctypes.c_void_p(out2.data_ptr()),
                                         ctypes.c_void_p(_stream_handle(stream)))
    if code != 0:
        raise TTALSError(code, "ttals_slice_error_noalloc", lib.ttals_last_error().decode())


def slice_error_noalloc_ptr(x_ptr: int, x_dtype: str, y_ptr: int, y_dtype: str, n: int, out2_ptr: int,
                            stream=None):
    """ttals_slice_error_noalloc on raw device pointers (see slice_error_noalloc)."""
    lib = load()
    code = lib.ttals_slice_error_noalloc(ctypes.c_void_p(x_ptr), DTYPES[x_dtype], ctypes.c_void_p(y_ptr),
                                         DTYPES[y_dtype], ctypes.c_int64(n), ctypes.c_void_p(out2_ptr),
                                         ctypes.c_void_p(_stream_handle(stream)))
    if code != 0:
        raise TTALSError(code, "ttals_slice_error_noalloc", lib.ttals_last_error().decode())
