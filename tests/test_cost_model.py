"""The tile cost model behind the decision not to build a degree-level
Karatsuba step on the tensor path (Sec. 4), checked against brute force and
closed forms (no GPU): a tile of a linear product is counted exactly when
one of its Toeplitz entries is nonzero; the direct kernels' MAC slots are
n^2 per digit pair times the N padding; the linear product's tiles cover all
m^2 of its nonzero entries; one block per product gives the 3/2 ratio."""
import numpy as np
import pytest

import bench


def _tile_nonzero_brute(m, blocks, k0):
    j = np.concatenate([np.arange(1024 * o, 1024 * o + 1024) for o in blocks])[:, None]
    k = np.arange(k0, k0 + 16)[None, :]
    d = j - k
    return bool(((d >= 0) & (d <= m - 1) & (k < m)).any())


@pytest.mark.parametrize("m,shifts", [(512, 1), (1024, 1), (1024, 2), (2048, 2)])
def test_linear_tile_predicate_against_brute_force(m, shifts):
    nblk = max(1, 2 * m // 1024)
    count = 0
    for g in range(0, nblk, shifts):
        blocks = range(g, min(nblk, g + shifts))
        for c in range(m // 16):
            want = _tile_nonzero_brute(m, blocks, 16 * c)
            assert bench._linear_tile_needed(m, blocks, 16 * c) == want, (m, g, c)
            count += want
    assert bench._linear_tiles(m, shifts) == count


@pytest.mark.parametrize("name,n,q,la,lb,s,tern", bench.KARATSUBA_SHAPES)
def test_direct_slots_closed_form(name, n, q, la, lb, s, tern):
    d = bench.karatsuba_model(n, q, la, lb, s, tern)["direct"]
    pad = d["mma_n"] / (8 * lb * s)
    assert d["mac_slots"] == la * lb * max(n, 1024) * n * pad


@pytest.mark.parametrize("m", [512, 2048, 8192])
def test_linear_tiles_cover_the_product(m):
    # every one of the m^2 nonzero entries lies in a counted tile of 1024 x 16
    assert bench._linear_tiles(m, 1) * 1024 * 16 >= m * m
    # and the skipped tiles are at least the two corner triangles' whole tiles
    assert bench._linear_tiles(m, 1) <= max(1, 2 * m // 1024) * (m // 16)


def test_one_block_ratio_and_widening():
    r = bench.karatsuba_model(1024, 12289, 2, 2, 1)
    k = r["karatsuba_shifts_1"]
    assert k["tiles_per_linear_product"] == 512 // 16 and k["mac_slot_ratio"] == 1.5
    # a 31-bit modulus: sums of two centred residues need a fifth 8-bit digit
    r = bench.karatsuba_model(4096, (1 << 31) - 1, 4, 4, 2)
    assert r["h1_digits"] == [5, 5]
    assert bench.karatsuba_model(4096, (1 << 31) - 1, 1, 4, 1, ternary_b=True)["h1_digits"] == [1, 5]
