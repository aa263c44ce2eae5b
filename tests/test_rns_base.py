"""The residue number system of small moduli that the tensor path's RNS
kernel uses (Sec. 2.4; RNS-base selection of the key-parameter section),
checked on the host against its definition with exact integers: odd,
pairwise coprime moduli below 2^8, each small enough that n ((m-1)/2)^2 <=
2^24 keeps fp32 sums of centred residues exact, taken largest first, and
just enough of them that their product exceeds 16 n floor(q/2)^2 (the range
of the centred integer products, with the reconstruction's margin)."""
import math

import pytest


@pytest.fixture(scope="module")
def pm():
    from paper_2307_06554_gb300 import build
    build.build()
    from paper_2307_06554_gb300 import polymul
    return polymul


def _cap(n):
    h = 0
    while (h + 1) ** 2 * n <= 1 << 24:
        h += 1
    return min(255, 2 * h + 1)


SHAPES = [(64, 3329), (256, 3329), (1024, 12289), (1024, (1 << 30) - 35), (2048, (1 << 31) - 1),
          (4096, (1 << 59) - 55), (1024, (1 << 62) - 57), (16384, (1 << 30) - 35), (8192, 65537)]


@pytest.mark.parametrize("n,q", SHAPES)
def test_base_definition(pm, n, q):
    ms = pm.polymul_tensor_rns_base(n, q)
    bound = 16 * n * (q // 2) ** 2
    assert 1 <= len(ms) <= 32
    assert ms == sorted(ms, reverse=True)
    for m in ms:
        assert m % 2 == 1 and 3 <= m <= _cap(n) < 256
        assert n * ((m - 1) // 2) ** 2 <= 1 << 24
    for i in range(len(ms)):
        for j in range(i):
            assert math.gcd(ms[i], ms[j]) == 1
    assert math.prod(ms) > bound
    assert math.prod(ms[:-1]) <= bound  # no more moduli than needed


@pytest.mark.parametrize("n,q", SHAPES)
def test_base_is_greedy_largest_first(pm, n, q):
    """Every odd candidate between the smallest chosen modulus and the cap
    that was skipped shares a factor with a larger chosen one."""
    ms = pm.polymul_tensor_rns_base(n, q)
    chosen = set(ms)
    for m in range(_cap(n), ms[-1], -2):
        if m not in chosen:
            assert any(math.gcd(m, x) > 1 for x in ms if x > m), m


def test_base_errors(pm):
    with pytest.raises(pm.PolymulError) as ei:
        pm.polymul_tensor_rns_base(8192, (1 << 59) - 55)  # 59-bit moduli at 2^13: moduli <= 91 do not reach 2^135
    assert ei.value.code == pm.POLYMUL_ENOTSUP
    for n, q in ((32, 12289), (1000, 12289), (32768, 12289), (1024, 1)):
        with pytest.raises(pm.PolymulError) as ei:
            pm.polymul_tensor_rns_base(n, q)
        assert ei.value.code == pm.POLYMUL_EINVAL, (n, q)


def test_caps_per_degree(pm):
    """The per-degree modulus cap: 255 up to n = 1024, then the largest odd
    m with n ((m-1)/2)^2 <= 2^24."""
    got = {n: max(pm.polymul_tensor_rns_base(n, 3)) for n in (64, 1024, 2048, 4096, 8192, 16384)}
    assert got == {64: 255, 1024: 255, 2048: 181, 4096: 129, 8192: 91, 16384: 65}
