"""Shared helpers for the GPU parity tests (no method arithmetic here)."""
import numpy as np


def to_dev(x: np.ndarray, device="cuda:0"):
    import torch
    if x.dtype == np.uint32:
        t = torch.from_numpy(np.ascontiguousarray(x).view(np.int32))
    elif x.dtype == np.uint64:
        t = torch.from_numpy(np.ascontiguousarray(x).view(np.int64))
    else:
        raise TypeError(x.dtype)
    return t.to(device)


def from_dev(t, dtype) -> np.ndarray:
    return t.cpu().numpy().view(dtype)


def run_plan_batch(plan, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    import torch
    ta, tb = to_dev(a), to_dev(b)
    tc = torch.full_like(ta, -1)
    plan.batch(ta, tb, tc)
    torch.cuda.synchronize()
    return from_dev(tc, a.dtype)


def assert_equal_residues(got: np.ndarray, want: np.ndarray, what: str = ""):
    got64 = got.astype(np.uint64)
    want64 = np.asarray(want).astype(np.uint64)
    if not np.array_equal(got64, want64):
        bad = np.argwhere(got64 != want64)
        i = tuple(bad[0])
        raise AssertionError("%s: %d mismatches, first at %s: got %d want %d"
                             % (what, len(bad), i, int(got64[i]), int(want64[i])))
