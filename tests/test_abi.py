"""The C-ABI library loads and exports every symbol include/polymul.h
declares; argument errors are reported without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(polymul_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2307_06554_gb300 import build
    build.build()
    from paper_2307_06554_gb300 import polymul
    return polymul


def test_header_declares_entry_points():
    names = _declared()
    for must in ("polymul_create", "polymul_batch", "polymul_destroy", "polymul_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(lib.library_path())
    missing = [n for n in _declared() if not hasattr(raw, n)]
    assert not missing, missing


@pytest.mark.parametrize("n,qs", [(100, [97]), (8, [97]), (131072, [97]), (1024, []), (1024, [1]),
                                  (1024, [12289, 12289]), (1024, [1 << 62])])
def test_create_rejects_bad_arguments(lib, n, qs):
    if not qs:
        # k = 0
        out = ctypes.c_void_p()
        rc = lib.lib().polymul_create(n, None, 0, None, ctypes.byref(out))
        assert rc == lib.POLYMUL_EINVAL
        return
    with pytest.raises(lib.PolymulError) as ei:
        lib.polymul_create(n, qs)
    assert ei.value.code == lib.POLYMUL_EINVAL
    assert lib.polymul_last_error()


def test_null_plan_calls(lib):
    L = lib.lib()
    assert L.polymul_batch(None, None, None, None, 1, None) == lib.POLYMUL_EINVAL
    assert L.polymul_batch_host(None, None, None, None, 1, None) == lib.POLYMUL_EINVAL
    assert L.polymul_batch_mapped(None, None, None, None, 1, None) == lib.POLYMUL_EINVAL
    L.polymul_destroy(None)  # no-op
    assert L.polymul_plan_info_get(None, None) == lib.POLYMUL_EINVAL


def test_null_handles_of_lists_and_servers(lib):
    """Entry points on uneven lists and servers report a NULL handle as
    EINVAL without touching a GPU."""
    L = lib.lib()
    assert L.polymul_ragged_select(None, 0) == lib.POLYMUL_EINVAL
    assert L.polymul_ragged_status(None, None) == lib.POLYMUL_EINVAL
    assert L.polymul_ragged_run(None, None, None, None, None) == lib.POLYMUL_EINVAL
    assert L.polymul_server_set_path(None, lib.PATH_TENSOR) == lib.POLYMUL_EINVAL
    assert L.polymul_server_set_route(None, lib.ROUTE_STAGED) == lib.POLYMUL_EINVAL
    assert L.polymul_plan_select(None, 0) == lib.POLYMUL_EINVAL


def test_replay_requests_are_marshalled_once(lib):
    """Server.prepare builds a replay's request structures ahead of time
    (outside any timed region): each carries the degree, the prime count,
    the prime indices and the operands' addresses, and replay accepts the
    prepared form (host logic only; nothing is submitted here)."""
    import numpy as np
    a = np.zeros((3, 64), np.uint64)
    b = np.ones((3, 64), np.uint64)
    c = np.empty((3, 64), np.uint64)
    arr, m, keep = lib.Server.prepare([(64, [0, 5, 9], a, b, c), (64, [2], a[:1], b[:1], c[:1])])
    assert m == 2 and len(keep) == 2
    assert (arr[0].n, arr[0].k, arr[1].k) == (64, 3, 1)
    assert [arr[0].prime_idx[i] for i in range(3)] == [0, 5, 9]
    assert arr[0].a == a.ctypes.data and arr[0].b == b.ctypes.data and arr[0].c == c.ctypes.data
