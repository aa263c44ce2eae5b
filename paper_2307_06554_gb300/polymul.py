"""Thin ctypes binding of libpolymul (include/polymul.h).

Argument marshalling only: every computation happens in the CUDA library.
Functions keep the C names (``polymul_create``, ``polymul_batch``, ...);
``Plan`` is a small convenience wrapper over them for torch tensors.
Importing this module loads the library and raises if it has not been
built (``python -c "import __graft_entry__ as g; g.build()"``); there is no
fallback of any kind.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

from . import build as _build

POLYMUL_OK = 0
POLYMUL_EINVAL = 1
POLYMUL_ENOTSUP = 2
POLYMUL_EDOMAIN = 3
POLYMUL_ENOMEM = 4
POLYMUL_ETIMEOUT = 5
POLYMUL_ECUDA = 6

PATH_AUTO = 0
PATH_NTT = 1
PATH_TENSOR = 2
FLAG_VALIDATE = 1
FLAG_TUNE = 2
FLAG_CYCLIC = 4  # the ring Z_q[x]/(x^n-1) instead of Z_q[x]/(x^n+1)
FLAG_TERNARY_B = 8  # b in {0, 1, q-1}: the tensor path takes b as one digit (c = b * T(a))
FLAG_OVERLAP = 16  # a batch may start while the previous batch launch on its stream drains
FLAG_HOST_STAGED = 32  # polymul_batch_host always copies through device staging buffers
ROUTE_DIRECT = 0  # server: mapped page-locked operands read and written in place (default)
ROUTE_STAGED = 1  # server: always copy through device memory

_ERRNAMES = {1: "EINVAL", 2: "ENOTSUP", 3: "EDOMAIN", 4: "ENOMEM", 5: "ETIMEOUT", 6: "ECUDA"}


class PolymulError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("polymul error %s (%d): %s" % (_ERRNAMES.get(code, "?"), code, msg))
        self.code = code


class polymul_opts(ctypes.Structure):
    _fields_ = [("path", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("tune_batch", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32 * 5)]


class polymul_plan_info(ctypes.Structure):
    _fields_ = [(name, ctypes.c_uint32) for name in
                ("n", "k", "elem_bytes", "path", "aux_primes", "block", "grid", "smem_bytes", "ctas_per_sm",
                 "digit_bits", "digits", "radix_bits", "candidates", "tuned", "tuned_batch",
                 "launch_flags", "ntt_mode", "regs", "cyclic", "tensor_groups", "rns_moduli",
                 "exchange_pad", "one_operand", "tensor_kernel", "kernel_regs", "kernel_max_block",
                 "host_direct")]


class polymul_tensor_shape_info(ctypes.Structure):
    _fields_ = [(name, ctypes.c_uint32) for name in
                ("kernel", "candidates", "digit_bits", "digits_a", "digits_b", "shifts", "slices", "groups",
                 "rns_moduli", "smem_bytes", "tmem_cols")] + [("reserved", ctypes.c_uint32 * 5)]


class polymul_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("k", ctypes.c_uint32), ("prime_offset", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("offset", ctypes.c_uint64)]


class polymul_request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("k", ctypes.c_uint32), ("prime_idx", ctypes.POINTER(ctypes.c_uint32)),
                ("a", ctypes.c_void_p), ("b", ctypes.c_void_p), ("c", ctypes.c_void_p)]


class polymul_server_stats(ctypes.Structure):
    _fields_ = [(x, ctypes.c_uint64) for x in ("submitted", "completed", "failed", "queued", "in_flight",
                                               "arena_bytes", "arena_peak_bytes")] + \
               [(x, ctypes.c_double) for x in ("p50_us", "p99_us", "mean_us", "max_us", "queue_p50_us",
                                               "queue_p99_us", "service_p50_us", "service_p99_us", "issue_us_mean",
                                               "server_busy_s")] + \
               [("completed_direct", ctypes.c_uint64)]


def library_path() -> str:
    """The in-tree build, or the file named by POLYMUL_LIB if set."""
    return os.environ.get("POLYMUL_LIB") or _build.LIB


def _load():
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError("libpolymul.so is not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    lib.polymul_create.argtypes = [u32, ctypes.POINTER(u64), u32, ctypes.POINTER(polymul_opts), ctypes.POINTER(vp)]
    lib.polymul_create.restype = i32
    lib.polymul_batch.argtypes = [vp, vp, vp, vp, u64, vp]
    lib.polymul_batch.restype = i32
    lib.polymul_batch_host.argtypes = [vp, vp, vp, vp, u64, vp]
    lib.polymul_batch_host.restype = i32
    lib.polymul_batch_mapped.argtypes = [vp, vp, vp, vp, u64, vp]
    lib.polymul_batch_mapped.restype = i32
    lib.polymul_batch_shared.argtypes = [vp, vp, vp, vp, u64, vp]
    lib.polymul_batch_shared.restype = i32
    lib.polymul_selftest_wait.argtypes = [ctypes.c_uint32, vp]
    lib.polymul_selftest_wait.restype = i32
    lib.polymul_tensor_rns_base.argtypes = [u32, u64, ctypes.POINTER(u32), u32, ctypes.POINTER(u32)]
    lib.polymul_tensor_rns_base.restype = i32
    lib.polymul_tensor_shape.argtypes = [u32, u64, u32, ctypes.POINTER(polymul_tensor_shape_info)]
    lib.polymul_tensor_shape.restype = i32
    lib.polymul_batch_static.argtypes = [u32, u64, vp, vp, vp, u64, vp]
    lib.polymul_batch_static.restype = i32
    lib.polymul_static_status.argtypes = [vp]
    lib.polymul_static_status.restype = i32
    lib.polymul_selftest_inject_wait.argtypes = [u32, u32]
    lib.polymul_selftest_inject_wait.restype = i32
    lib.polymul_plan_select.argtypes = [vp, u32]
    lib.polymul_plan_select.restype = i32
    lib.polymul_tune.argtypes = [vp, u64, vp]
    lib.polymul_tune.restype = i32
    lib.polymul_plan_status.argtypes = [vp, vp]
    lib.polymul_plan_status.restype = i32
    lib.polymul_plan_info_get.argtypes = [vp, ctypes.POINTER(polymul_plan_info)]
    lib.polymul_plan_info_get.restype = i32
    lib.polymul_destroy.argtypes = [vp]
    lib.polymul_destroy.restype = None
    lib.polymul_ragged_create.argtypes = [ctypes.POINTER(u64), u32, u32, ctypes.POINTER(vp)]
    lib.polymul_ragged_create.restype = i32
    lib.polymul_ragged_prepare.argtypes = [vp, ctypes.POINTER(polymul_desc), u32, ctypes.POINTER(u32), u64, u64,
                                           ctypes.POINTER(vp)]
    lib.polymul_ragged_prepare.restype = i32
    for name in ("polymul_ragged_run", "polymul_ragged_run_graph"):
        getattr(lib, name).argtypes = [vp, vp, vp, vp, vp]
        getattr(lib, name).restype = i32
    lib.polymul_ragged_status.argtypes = [vp, vp]
    lib.polymul_ragged_status.restype = i32
    lib.polymul_ragged_tune.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(u32)]
    lib.polymul_ragged_tune.restype = i32
    lib.polymul_ragged_select.argtypes = [vp, u32]
    lib.polymul_ragged_select.restype = i32
    lib.polymul_ragged_batch_info.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(u32)]
    lib.polymul_ragged_batch_info.restype = i32
    lib.polymul_ragged_batch_destroy.argtypes = [vp]
    lib.polymul_ragged_batch_destroy.restype = None
    lib.polymul_ragged_destroy.argtypes = [vp]
    lib.polymul_ragged_destroy.restype = None
    lib.polymul_server_create.argtypes = [ctypes.POINTER(u64), u32, u32, u64, u32, ctypes.POINTER(vp)]
    lib.polymul_server_create.restype = i32
    lib.polymul_server_submit.argtypes = [vp, ctypes.POINTER(polymul_request), ctypes.POINTER(u64)]
    lib.polymul_server_submit.restype = i32
    lib.polymul_server_poll.argtypes = [vp, u64, ctypes.POINTER(ctypes.c_int)]
    lib.polymul_server_set_path.restype = ctypes.c_int
    lib.polymul_server_set_path.argtypes = [vp, u32]
    lib.polymul_server_set_route.restype = ctypes.c_int
    lib.polymul_server_set_route.argtypes = [vp, u32]
    lib.polymul_server_poll.restype = i32
    lib.polymul_server_wait.argtypes = [vp, u64, ctypes.c_double]
    lib.polymul_server_wait.restype = i32
    lib.polymul_server_replay.argtypes = [vp, ctypes.POINTER(polymul_request), u32, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]
    lib.polymul_server_replay.restype = i32
    lib.polymul_server_stats_get.argtypes = [vp, ctypes.POINTER(polymul_server_stats), ctypes.c_int]
    lib.polymul_server_stats_get.restype = i32
    lib.polymul_server_destroy.argtypes = [vp]
    lib.polymul_server_destroy.restype = None
    lib.polymul_last_error.argtypes = []
    lib.polymul_last_error.restype = ctypes.c_char_p
    return lib


_lib = _load()


def lib():
    return _lib


def polymul_last_error() -> str:
    return _lib.polymul_last_error().decode()


def _check(rc: int):
    if rc != POLYMUL_OK:
        raise PolymulError(rc, polymul_last_error())


def _ptr(x) -> int:
    """Device/host address of a torch tensor, numpy array or raw integer."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError("cannot take the address of %r" % type(x))


def _stream(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def polymul_create(n: int, q_list: Sequence[int], path: int = PATH_AUTO, flags: int = 0,
                   tune_batch: int = 0) -> int:
    arr = (ctypes.c_uint64 * len(q_list))(*[int(q) for q in q_list])
    opts = polymul_opts(path, flags, tune_batch)
    out = ctypes.c_void_p()
    _check(_lib.polymul_create(n, arr, len(q_list), ctypes.byref(opts), ctypes.byref(out)))
    return out.value


def polymul_batch(plan: int, a, b, c, batch: int, stream=None) -> None:
    _check(_lib.polymul_batch(plan, _ptr(a), _ptr(b), _ptr(c), batch, _stream(stream)))


def polymul_batch_host(plan: int, a, b, c, batch: int, stream=None) -> None:
    _check(_lib.polymul_batch_host(plan, _ptr(a), _ptr(b), _ptr(c), batch, _stream(stream)))


def polymul_batch_mapped(plan: int, a, b, c, batch: int, stream=None) -> None:
    """a, b, c in page-locked host memory the device maps; asynchronous on
    `stream` (results in c once it has been synchronised)."""
    _check(_lib.polymul_batch_mapped(plan, _ptr(a), _ptr(b), _ptr(c), batch, _stream(stream)))


def polymul_selftest_wait(polls: int, stream=None) -> None:
    """Device check that a bounded wait gives up: raises PolymulError with
    POLYMUL_ETIMEOUT when it does (the expected outcome)."""
    _check(_lib.polymul_selftest_wait(polls, _stream(stream)))


def polymul_tensor_shape(n: int, qmax: int, flags: int = 0) -> dict:
    """The tensor path's default kernel for degree n and moduli up to qmax
    (host only; no plan is created)."""
    info = polymul_tensor_shape_info()
    _check(_lib.polymul_tensor_shape(n, qmax, flags, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in polymul_tensor_shape_info._fields_ if name != "reserved"}


def polymul_tensor_rns_base(n: int, qmax: int) -> list:
    """The small moduli of the tensor path's residue-number-system kernel
    for degree n and moduli up to qmax (host only)."""
    count = ctypes.c_uint32(0)
    _check(_lib.polymul_tensor_rns_base(n, qmax, None, 0, ctypes.byref(count)))
    out = (ctypes.c_uint32 * max(1, count.value))()
    _check(_lib.polymul_tensor_rns_base(n, qmax, out, count.value, ctypes.byref(count)))
    return [int(x) for x in out[:count.value]]


def polymul_batch_shared(plan: int, a, b, c, batch: int, stream=None) -> None:
    """c_i = a * b_i for one shared operand a ([k][n]) and b, c [batch][k][n]."""
    _check(_lib.polymul_batch_shared(plan, _ptr(a), _ptr(b), _ptr(c), batch, _stream(stream)))


def polymul_batch_static(n: int, q: int, a, b, c, batch: int, stream=None) -> None:
    """Allocation-free entry point (one NTT-friendly prime, n <= 4096)."""
    _check(_lib.polymul_batch_static(n, q, _ptr(a), _ptr(b), _ptr(c), batch, _stream(stream)))


def polymul_static_status(stream=None) -> None:
    """Raises PolymulError (POLYMUL_ETIMEOUT) when the last
    polymul_batch_static call on the current device abandoned a device wait."""
    _check(_lib.polymul_static_status(_stream(stream)))


def polymul_selftest_inject_wait(launches: int, polls: int) -> None:
    """Diagnostics: the next `launches` NTT batch-kernel launches take an
    expired bounded wait after `polls` polls (no device fault)."""
    _check(_lib.polymul_selftest_inject_wait(launches, polls))


def polymul_plan_select(plan: int, candidate: int) -> None:
    _check(_lib.polymul_plan_select(plan, candidate))


def polymul_tune(plan: int, batch: int, stream=None) -> None:
    _check(_lib.polymul_tune(plan, batch, _stream(stream)))


def polymul_plan_status(plan: int, stream=None) -> None:
    _check(_lib.polymul_plan_status(plan, _stream(stream)))


def polymul_plan_info_get(plan: int) -> dict:
    info = polymul_plan_info()
    _check(_lib.polymul_plan_info_get(plan, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in polymul_plan_info._fields_ if name != "reserved"}


def polymul_destroy(plan: int) -> None:
    _lib.polymul_destroy(plan)


class Plan:
    """Owning wrapper: ``with Plan(n, qs) as p: p.batch(a, b, c)``."""

    def __init__(self, n: int, q_list: Sequence[int], path: int = PATH_AUTO, flags: int = 0,
                 tune_batch: int = 0):
        self.n = int(n)
        self.q_list = [int(q) for q in q_list]
        self.handle = polymul_create(self.n, self.q_list, path, flags, tune_batch)
        self.info = polymul_plan_info_get(self.handle)

    def select(self, candidate: int) -> dict:
        polymul_plan_select(self.handle, candidate)
        self.info = polymul_plan_info_get(self.handle)
        return self.info

    def tune(self, batch: int, stream=None) -> dict:
        polymul_tune(self.handle, batch, stream)
        self.info = polymul_plan_info_get(self.handle)
        return self.info

    @property
    def elem_bytes(self) -> int:
        return self.info["elem_bytes"]

    def batch(self, a, b, c, stream=None) -> None:
        """a, b, c: device tensors of shape [batch][k][n] (uint32/int32 or
        uint64/int64 per elem_bytes)."""
        batch = self._check_shapes(a, b, c)
        polymul_batch(self.handle, a, b, c, batch, stream if stream is not None else _current_stream(a))

    def batch_host(self, a, b, c) -> None:
        batch = self._check_shapes(a, b, c)
        polymul_batch_host(self.handle, a, b, c, batch, None)

    def batch_mapped(self, a, b, c, stream=None) -> None:
        """a, b, c: page-locked host tensors [batch][k][n]; asynchronous."""
        batch = self._check_shapes(a, b, c)
        polymul_batch_mapped(self.handle, a, b, c, batch, stream)

    def _check_shapes(self, a, b, c) -> int:
        shape = tuple(a.shape)
        if tuple(b.shape) != shape or tuple(c.shape) != shape:
            raise ValueError("a, b, c must have the same shape")
        if len(shape) != 3 or shape[1] != len(self.q_list) or shape[2] != self.n:
            raise ValueError("expected shape [batch][%d][%d], got %s" % (len(self.q_list), self.n, shape))
        for x in (a, b, c):
            size = x.element_size() if hasattr(x, "element_size") else x.itemsize
            if size != self.elem_bytes:
                raise ValueError("element size must be %d bytes" % self.elem_bytes)
            contiguous = x.is_contiguous() if hasattr(x, "is_contiguous") else x.flags["C_CONTIGUOUS"]
            if not contiguous:
                raise ValueError("operands must be contiguous")
        return shape[0]

    def close(self):
        if self.handle:
            polymul_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _current_stream(x):
    try:
        import torch
        if isinstance(x, torch.Tensor) and x.is_cuda:
            return torch.cuda.current_stream(x.device).cuda_stream
    except ImportError:  # pragma: no cover
        pass
    return 0


# ---------------------------------------------------------------- uneven batches
def polymul_ragged_create(pool: Sequence[int], n_max: int) -> int:
    arr = (ctypes.c_uint64 * len(pool))(*[int(q) for q in pool])
    out = ctypes.c_void_p()
    _check(_lib.polymul_ragged_create(arr, len(pool), n_max, ctypes.byref(out)))
    return out.value


def polymul_ragged_prepare(ctx: int, descs: Sequence[tuple], prime_idx: Sequence[int], total_elems: int) -> int:
    """descs: (n, k, prime_offset, offset) per product."""
    d = (polymul_desc * max(1, len(descs)))(*[polymul_desc(n, k, po, 0, off) for (n, k, po, off) in descs])
    pi = (ctypes.c_uint32 * max(1, len(prime_idx)))(*[int(x) for x in prime_idx])
    out = ctypes.c_void_p()
    _check(_lib.polymul_ragged_prepare(ctx, d, len(descs), pi, len(prime_idx), total_elems, ctypes.byref(out)))
    return out.value


def polymul_ragged_run(batch: int, a, b, c, stream=None) -> None:
    _check(_lib.polymul_ragged_run(batch, _ptr(a), _ptr(b), _ptr(c), _stream(stream)))


def polymul_ragged_run_graph(batch: int, a, b, c, stream=None) -> None:
    _check(_lib.polymul_ragged_run_graph(batch, _ptr(a), _ptr(b), _ptr(c), _stream(stream)))


def polymul_ragged_status(batch: int, stream=None) -> None:
    _check(_lib.polymul_ragged_status(batch, _stream(stream)))


# polymul_ragged_select / _tune choice bits: bit 0 the shape set of degrees
# 2^10..2^13, bit 1 that of 2^14, bit 2 + (log2 n - 10) degree class n on
# the tensor path
RAGGED_TENSOR_SHIFT = 2


def ragged_tensor_bits(*logns) -> int:
    """Choice bits putting the degree classes 2^logn on the tensor path."""
    return sum(1 << (RAGGED_TENSOR_SHIFT + l - 10) for l in logns)


def polymul_ragged_tune(batch: int, a, b, c, stream=None) -> int:
    """Pick each launch's shape set, then each degree class's path, by
    measurement; returns the choice bits (see RAGGED_TENSOR_SHIFT)."""
    ch = ctypes.c_uint32(0)
    _check(_lib.polymul_ragged_tune(batch, _ptr(a), _ptr(b), _ptr(c), _stream(stream), ctypes.byref(ch)))
    return ch.value


def polymul_ragged_batch_info(batch: int) -> dict:
    u, i, g = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint32()
    _check(_lib.polymul_ragged_batch_info(batch, ctypes.byref(u), ctypes.byref(i), ctypes.byref(g)))
    return {"units": u.value, "items": i.value, "grid": g.value}


def polymul_ragged_batch_destroy(batch: int) -> None:
    _lib.polymul_ragged_batch_destroy(batch)


def polymul_ragged_destroy(ctx: int) -> None:
    _lib.polymul_ragged_destroy(ctx)


class Ragged:
    """Owning wrapper for a prime pool plus one prepared list of products.

    ``layout(products)`` assigns offsets; ``run(a, b, c)`` launches once."""

    def __init__(self, pool: Sequence[int], n_max: int, products: Sequence[tuple]):
        """products: (n, [pool indices]) per product, packed back to back."""
        self.ctx = polymul_ragged_create(pool, n_max)
        descs, prime_idx, off = [], [], 0
        for n, idx in products:
            descs.append((n, len(idx), len(prime_idx), off))
            prime_idx.extend(idx)
            off += n * len(idx)
        self.total = off
        self.offsets = [d[3] for d in descs]
        try:
            self.batch = polymul_ragged_prepare(self.ctx, descs, prime_idx, off)
        except Exception:
            polymul_ragged_destroy(self.ctx)
            raise
        self.info = polymul_ragged_batch_info(self.batch)

    def run(self, a, b, c, stream=None, graph=False):
        (polymul_ragged_run_graph if graph else polymul_ragged_run)(self.batch, a, b, c, stream)

    def tune(self, a, b, c, stream=None) -> int:
        return polymul_ragged_tune(self.batch, a, b, c, stream)

    def select(self, choice: int) -> None:
        _check(_lib.polymul_ragged_select(self.batch, choice))

    def close(self):
        if getattr(self, "batch", None):
            polymul_ragged_batch_destroy(self.batch)
            self.batch = None
        if getattr(self, "ctx", None):
            polymul_ragged_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---------------------------------------------------------------- serving
class Server:
    """Continuously batching request loop (see polymul_server_* in the
    header).  Operands are host numpy uint64 arrays of shape [k][n]; keep
    them alive until the request completes."""

    def __init__(self, pool: Sequence[int], n_max: int, device_bytes: int = 1 << 30, lanes: int = 8):
        arr = (ctypes.c_uint64 * len(pool))(*[int(q) for q in pool])
        out = ctypes.c_void_p()
        _check(_lib.polymul_server_create(arr, len(pool), n_max, device_bytes, lanes, ctypes.byref(out)))
        self.handle = out.value
        self._keep = {}

    @staticmethod
    def _req(n, prime_idx, a, b, c):
        idx = (ctypes.c_uint32 * len(prime_idx))(*[int(x) for x in prime_idx])
        r = polymul_request(n, len(prime_idx), idx, _ptr(a), _ptr(b), _ptr(c))
        return r, idx

    def submit(self, n, prime_idx, a, b, c) -> int:
        r, idx = self._req(n, prime_idx, a, b, c)
        t = ctypes.c_uint64()
        _check(_lib.polymul_server_submit(self.handle, ctypes.byref(r), ctypes.byref(t)))
        return t.value

    def set_path(self, path: int) -> None:
        """Path of the requests submitted from now on (PATH_NTT or PATH_TENSOR)."""
        _check(_lib.polymul_server_set_path(self.handle, path))

    def set_route(self, route: int) -> None:
        """Host route of the requests submitted from now on (ROUTE_DIRECT or
        ROUTE_STAGED)."""
        _check(_lib.polymul_server_set_route(self.handle, route))

    def poll(self, ticket: int) -> bool:
        d = ctypes.c_int()
        _check(_lib.polymul_server_poll(self.handle, ticket, ctypes.byref(d)))
        return bool(d.value)

    def wait(self, ticket: int, timeout_s: float = 60.0) -> None:
        _check(_lib.polymul_server_wait(self.handle, ticket, timeout_s))

    @staticmethod
    def prepare(requests):
        """The request array of a replay, built once: (n, prime_idx, a, b, c)
        tuples marshalled into polymul_request structures (the operands are
        referenced, not copied)."""
        m = len(requests)
        arr = (polymul_request * max(1, m))()
        keep = []
        for i, (n, idx, a, b, c) in enumerate(requests):
            r, ix = Server._req(n, idx, a, b, c)
            arr[i] = r
            keep.append(ix)
        return (arr, m, keep)

    def replay(self, requests, arrival_s):
        """requests: (n, prime_idx, a, b, c) tuples, or what prepare()
        returned for them; returns latencies (us)."""
        arr, m, _keep = requests if isinstance(requests, tuple) else self.prepare(requests)
        times = (ctypes.c_double * max(1, m))(*[float(x) for x in arrival_s])
        lat = (ctypes.c_double * max(1, m))()
        _check(_lib.polymul_server_replay(self.handle, arr, m, times, lat))
        return [lat[i] for i in range(m)]

    def stats(self, reset: bool = False) -> dict:
        st = polymul_server_stats()
        _check(_lib.polymul_server_stats_get(self.handle, ctypes.byref(st), int(reset)))
        return {name: getattr(st, name) for name, _ in polymul_server_stats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            _lib.polymul_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
