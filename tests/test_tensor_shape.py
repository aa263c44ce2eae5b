"""Host-side shape selection of the tensor path (polymul_tensor_shape; no
GPU needed), checked against its definitions with exact integers: the digit
width keeps every fp32 partial sum exact (n 2^(2w-2) <= 2^24) and every
digit exact in bf16 (|d| <= 2^(w-1) <= 128); L balanced digits in
[-2^(w-1), 2^(w-1)) reach floor(q/2) -- their positive reach is
(2^(w-1) - 1)(2^(wL) - 1)/(2^w - 1), less than (2^(wL) - 1)/2, which moduli
just below a boundary expose; every returned configuration fits the
hardware (shared memory per CTA, tensor-memory columns); the bench's
mirrored formulas agree with the library."""
import math

import pytest


@pytest.fixture(scope="module")
def pm():
    from paper_2307_06554_gb300 import build
    build.build()
    from paper_2307_06554_gb300 import polymul
    return polymul


def _width(n):
    return min(8, (24 - (n.bit_length() - 1)) // 2 + 1)


def _reach(w, L):
    return ((1 << (w - 1)) - 1) * ((1 << (w * L)) - 1) // ((1 << w) - 1)


def _digits(n, q):
    w = _width(n)
    return w, next(L for L in range(1, 9) if _reach(w, L) >= q // 2)


def _drain_digits(q):
    """8-bit digits of the drained kernel (exact per K chunk of 1024 at any
    degree), at most four; None past that."""
    return next((L for L in range(1, 5) if _reach(8, L) >= q // 2), None)


def _drain_digits64(q):
    return next(L for L in range(1, 9) if _reach(8, L) >= q // 2)


def _default_digits(n, q):
    """The default digit kernel's (width, digits): the drained one where
    the undrained width is below 8 and it needs fewer digits, or where the
    undrained one has none (more than five digits)."""
    w, L = _digits(n, q)
    l8 = _drain_digits(q)
    if w < 8 and l8 is not None and (l8 < L or L > 5):
        return 8, l8
    return w, L


def test_reach_is_the_balanced_digit_range():
    """Brute force on small widths: the largest value L balanced w-bit digits
    represent is the closed form used above."""
    for w in (2, 3, 4):
        for L in (1, 2, 3):
            vals = {0}
            for _ in range(L):
                vals = {v * (1 << w) + d for v in vals for d in range(-(1 << (w - 1)), 1 << (w - 1))}
            assert max(vals) == _reach(w, L)
            assert min(vals) == -(1 << (w - 1)) * ((1 << (w * L)) - 1) // ((1 << w) - 1)


@pytest.mark.parametrize("n,q,digits", [(1024, 65521, 3), (1024, 65279, 2), (1024, 65281, 3), (2048, 16381, 3),
                                        (2048, 16253, 2), (4096, 16383, 3), (1024, 12289, 2), (256, 3329, 2),
                                        (4096, 1073479681, 5)])
def test_digit_boundaries(pm, n, q, digits):
    assert digits == _digits(n, q)[1]
    info = pm.polymul_tensor_shape(n, q)
    assert (info["digit_bits"], info["digits_b"]) == _default_digits(n, q)
    assert info["digits_a"] == info["digits_b"]
    assert info["kernel"] == (4 if info["digit_bits"] != _width(n) else 1 if n == 1024 else 2)


def test_more_than_five_digits_go_to_the_drained_kernel(pm):
    info = pm.polymul_tensor_shape(8192, 1073479681)  # needs six digits of 6 bits
    assert _digits(8192, 1073479681)[1] == 6
    assert (info["kernel"], info["digit_bits"], info["digits_b"], info["candidates"]) == (4, 8, 4, 3)
    # a 32-bit word modulus above 2^31: the RNS kernel alone
    info = pm.polymul_tensor_shape(8192, 2147483659)
    assert info["kernel"] == 3 and info["rns_moduli"] == len(pm.polymul_tensor_rns_base(8192, 2147483659))


def test_sweep_fits_the_hardware(pm):
    """Every degree and a spread of modulus sizes: the exactness bounds, and
    shared memory and tensor memory within one CTA's limits."""
    seen = set()
    for logn in range(6, 15):
        n = 1 << logn
        for bits in (2, 5, 8, 12, 14, 17, 20, 24, 28, 30, 31, 32, 40, 50, 59, 61):
            q = (1 << bits) - 1 if bits < 62 else (1 << 61) + 1
            for flags in (0, pm.FLAG_TERNARY_B):
                try:
                    info = pm.polymul_tensor_shape(n, q, flags)
                except pm.PolymulError as e:
                    assert e.code == pm.POLYMUL_ENOTSUP
                    continue
                seen.add(info["kernel"])
                assert info["smem_bytes"] <= 227 * 1024 and info["tmem_cols"] <= 512
                assert info["tmem_cols"] >= 32 and info["tmem_cols"] & (info["tmem_cols"] - 1) == 0
                if info["kernel"] == 6:
                    # 64-bit words: drained 8-bit digits, at least five
                    assert info["digit_bits"] == 8 and q >= 1 << 32 and n >= 1024
                    assert info["digits_a"] == info["digits_b"] == max(5, _drain_digits64(q))
                elif info["kernel"] in (1, 2, 4):
                    w = info["digit_bits"]
                    # exact fp32 sums over the whole of K, or over chunks of
                    # at most 1024 for the drained kernel
                    assert min(n, 1024 if info["kernel"] == 4 else n) * (1 << (2 * w - 2)) <= 1 << 24
                    assert (1 << (w - 1)) <= 128
                    assert (w, info["digits_b"]) == _default_digits(n, q)
                    assert q < 1 << 31
                else:
                    ms = pm.polymul_tensor_rns_base(n, q)
                    assert info["rns_moduli"] == len(ms)
                    assert math.prod(ms) > 16 * n * (q // 2) ** 2
                    assert info["rns_moduli"] * max(16, 8 * info["shifts"]) <= 512
                blocks = max(1, n // 1024)
                assert info["groups"] == 0 or info["groups"] * info["shifts"] * info["slices"] == blocks
    assert seen == {1, 2, 3, 4, 6}


def test_kernel_choice(pm):
    assert pm.polymul_tensor_shape(1024, 12289)["kernel"] == 1          # whole product first at 1024
    i = pm.polymul_tensor_shape(2048, 12289)
    assert (i["kernel"], i["shifts"], i["groups"]) == (2, 2, 1)          # shifted copies of b at 2048
    i = pm.polymul_tensor_shape(4096, (1 << 30) - 35, pm.FLAG_TERNARY_B)
    assert (i["kernel"], i["digits_a"], i["digits_b"], i["shifts"], i["slices"]) == (4, 1, 4, 1, 4)
    i = pm.polymul_tensor_shape(4096, (1 << 30) - 35)
    assert (i["kernel"], i["digits_a"], i["digits_b"], i["shifts"], i["groups"]) == (4, 4, 4, 2, 2)
    i = pm.polymul_tensor_shape(16384, (1 << 31) - 1)   # six 6-bit digits undrained: drained only
    assert (i["kernel"], i["digits_b"], i["candidates"]) == (4, 4, 2)
    i = pm.polymul_tensor_shape(4096, (1 << 59) - 55)
    assert (i["kernel"], i["rns_moduli"], i["shifts"], i["groups"]) == (3, 21, 2, 2)
    i = pm.polymul_tensor_shape(8192, (1 << 59) - 55)   # no RNS base: the 64-bit digit kernel
    assert (i["kernel"], i["digits_a"], i["digits_b"], i["groups"]) == (6, 8, 8, 8)
    i = pm.polymul_tensor_shape(65536, (1 << 59) - 55)
    assert (i["kernel"], i["groups"], i["candidates"]) == (6, 64, 1)
    i = pm.polymul_tensor_shape(1024, (1 << 59) - 55)   # first up to n = 2048
    assert (i["kernel"], i["candidates"]) == (6, 2)
    for n, q in ((32768, 12289), (16, 12289), (32768, (1 << 30) - 35)):
        with pytest.raises(pm.PolymulError) as ei:
            pm.polymul_tensor_shape(n, q)
        assert ei.value.code == pm.POLYMUL_ENOTSUP, (n, q)
    with pytest.raises(pm.PolymulError) as ei:
        pm.polymul_tensor_shape(1000, 12289)
    assert ei.value.code == pm.POLYMUL_EINVAL


def test_bench_mirrors_agree(pm):
    """bench.py derives its shared-memory rooflines from the digit count and
    the shift counts; its formulas must match the library's choices."""
    import bench
    for logn in range(6, 15):
        n = 1 << logn
        for q in (3329, 12289, 65521, 1000003, (1 << 30) - 35, (1 << 59) - 55):
            try:
                info = pm.polymul_tensor_shape(n, q)
            except pm.PolymulError:
                continue
            if info["kernel"] == 3:
                assert bench._rns_shifts(n, info["rns_moduli"]) == info["shifts"], (n, q)
            else:
                if info["kernel"] in (1, 2):
                    assert bench._tensor_digits(n, q) == (info["digit_bits"], info["digits_b"]), (n, q)
                if info["kernel"] in (2, 4):
                    got = bench._tiled_shifts(n, {"tensor_groups": info["groups"]})
                    assert got == info["shifts"], (n, q)
