"""ctypes driver for the plain C schoolbook oracle (``schoolbook.c``).

TEST INFRASTRUCTURE ONLY (tests, smoke(), bench.py's CPU baseline).
``build()`` compiles the C file with the host gcc into ``oracle/_build``;
the batch driver splits products over host threads (ctypes releases the
GIL for the duration of each foreign call, so threads run in parallel).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "schoolbook.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile schoolbook.c (portable C, no target-specific flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64p = ctypes.POINTER(ctypes.c_uint64)
            for fn in (lib.oracle_negacyclic_batch, lib.oracle_cyclic_batch):
                fn.argtypes = [u64p, u64p, u64p, ctypes.c_uint64, u64p, ctypes.c_uint64, ctypes.c_uint64,
                               ctypes.c_uint64]
                fn.restype = None
            for fn in (lib.oracle_negacyclic_coeffs, lib.oracle_cyclic_coeffs):
                fn.argtypes = [u64p, u64p, ctypes.c_uint64, ctypes.c_uint64, u64p, ctypes.c_uint64, u64p]
                fn.restype = None
            _lib = lib
    return _lib


def _ptr(x: np.ndarray):
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)


def polymul_batch(a: np.ndarray, b: np.ndarray, q_list: Sequence[int],
                  threads: Optional[int] = None, cyclic: bool = False) -> np.ndarray:
    """Oracle over a [batch][k][n] batch; returns uint64 [batch][k][n].
    ``cyclic``: the ring Z_q[x]/(x^n-1) instead of Z_q[x]/(x^n+1)."""
    if a.shape != b.shape or a.ndim != 3 or a.shape[1] != len(q_list):
        raise ValueError("shape mismatch")
    lib = _load()
    a64 = np.ascontiguousarray(a, dtype=np.uint64)
    b64 = np.ascontiguousarray(b, dtype=np.uint64)
    c64 = np.zeros_like(a64)
    qs = np.ascontiguousarray(np.asarray(q_list, dtype=np.uint64))
    batch, k, n = a64.shape
    threads = threads or default_threads()
    threads = max(1, min(threads, batch))
    chunks = []
    step = (batch + threads - 1) // threads
    for first in range(0, batch, step):
        chunks.append((first, min(step, batch - first)))

    fn = lib.oracle_cyclic_batch if cyclic else lib.oracle_negacyclic_batch

    def run(ch):
        fn(_ptr(a64), _ptr(b64), _ptr(c64), n, _ptr(qs), k, ch[0], ch[1])

    if len(chunks) == 1:
        run(chunks[0])
    else:
        with ThreadPoolExecutor(max_workers=len(chunks)) as ex:
            list(ex.map(run, chunks))
    return c64


def polymul_one(a: np.ndarray, b: np.ndarray, q: int, cyclic: bool = False) -> np.ndarray:
    """One product of two length-n residue vectors."""
    r = polymul_batch(np.asarray(a).reshape(1, 1, -1), np.asarray(b).reshape(1, 1, -1), [q], threads=1,
                      cyclic=cyclic)
    return r[0, 0]


def coeffs(a: np.ndarray, b: np.ndarray, q: int, js: Sequence[int], cyclic: bool = False) -> np.ndarray:
    """Selected output coefficients c_j of one product (sampled checks at
    sizes where the whole product would take too long)."""
    lib = _load()
    a64 = np.ascontiguousarray(a, dtype=np.uint64).reshape(-1)
    b64 = np.ascontiguousarray(b, dtype=np.uint64).reshape(-1)
    jj = np.ascontiguousarray(np.asarray(js, dtype=np.uint64))
    out = np.zeros(len(jj), dtype=np.uint64)
    fn = lib.oracle_cyclic_coeffs if cyclic else lib.oracle_negacyclic_coeffs
    fn(_ptr(a64), _ptr(b64), a64.size, int(q), _ptr(jj), len(jj), _ptr(out))
    return out
