"""Host-side checks of the qubit grouping behind the streaming passes (Sec. 2.3
layers applied group by group), through z2_plan_geometry: no GPU needed.

Every qubit must be rotated by exactly one group; each group's tile must hold
its passenger bits and its rotated bits; and the 5-D TMA view the ring kernel
uses for a group (rows, tile-id range, rotated range(s), tile-id range) must
address exactly the tile's amplitudes, inside the state, with the tile bits in
the order the kernel assumes.  The view is rebuilt here from the group
description alone, following the layout stated in include/z2lgt.h.
"""
import pytest

import paper_1910_08020_gb300 as z2

SPREAD_BITS = 21  # rows less than 16 MB (2^21 complex64 amplitudes) apart


def rotated_bits(g, low):
    if low:
        return list(range(g.k))
    bits = list(range(g.b, g.b + g.k1))
    if g.k1 < g.k:
        bits += list(range(g.b2, g.b2 + g.k - g.k1))
    return bits


def tile_bits_in_order(g):
    """Global bit of each tile bit, as the kernel numbers them (passengers first)."""
    return list(range(g.c)) + ([] if g.c == g.tile_bits else rotated_bits(g, False))


def tma_view(n, g):
    """(dims, element strides of dims 1..4, box) of the ring kernel's view."""
    if g.k1 < g.k:
        c, b, k1, k2, b2 = g.c, g.b, g.k1, g.k - g.k1, g.b2
        return ([1 << c, 1 << (b - c), 1 << k1, 1 << (b2 - b - k1), 1 << k2],
                [1 << c, 1 << b, 1 << (b + k1), 1 << b2], [1 << c, 1, 1 << k1, 1, 1 << k2])
    cp, bp = g.c, g.b
    if cp > 8:  # contiguous tile viewed as 2^8 x 2^(tb - 8)
        cp = bp = 8
    k = g.tile_bits - cp
    k1, k2 = min(k, 8), k - min(k, 8)
    return ([1 << cp, 1 << (bp - cp), 1 << k1, 1 << k2, 1 << (n - bp - k)],
            [1 << cp, 1 << bp, 1 << (bp + k1), 1 << (bp + k)], [1 << cp, 1, 1 << k1, 1 << k2, 1])


def log2(v):
    assert v > 0 and v & (v - 1) == 0
    return v.bit_length() - 1


def check_plan(n, tile_bits, variant, tma):
    groups = z2.z2_plan_geometry(n, 0, tile_bits, variant, tma)
    covered = []
    for i, g in enumerate(groups):
        low = i == 0
        covered += rotated_bits(g, low)
        if len(groups) == 1:
            assert g.tile_bits == n and g.c == n and g.k == n
            continue
        if low:
            assert g.c == g.b == g.tile_bits and 1 <= g.k <= g.tile_bits
        else:
            assert g.c + g.k == g.tile_bits, "a strided tile is its passengers plus its rotated bits"
            # at least 3 passenger bits (64-byte rows), except the 24-qubit ring
            # rule's 2 (32-byte rows, on a state about the size of L2)
            assert (g.c >= 3 or (n == 24 and g.c == 2 and g.tile_bits == 13)) and g.c <= 8 and g.b >= g.c
            if g.k1 < g.k:
                assert 1 <= g.k1 <= 8 and 1 <= g.k - g.k1 <= 8
                assert g.b2 >= g.b + g.k1 and g.b2 + g.k - g.k1 == n, "the upper range ends at the top bit"
        dims, strides, box = tma_view(n, g)
        assert all(x <= 256 for x in box) and (box[0] * 8) % 16 == 0
        # box order (dim 0 fastest) must list the tile bits in the kernel's order
        order = []
        for d in range(5):
            base = 0 if d == 0 else log2(strides[d - 1])
            order += [base + j for j in range(log2(box[d]))]
        assert order == tile_bits_in_order(g)
        # the dims with box 1 carry the tile id; with the tile bits they cover the state once
        id_bits = []
        for d in range(1, 5):
            if box[d] == 1 and dims[d] > 1:
                id_bits += [log2(strides[d - 1]) + j for j in range(log2(dims[d]))]
        assert sorted(order + id_bits) == list(range(n))
        for d in range(5):
            assert box[d] == dims[d] or box[d] == 1
        last = sum((dims[d] - 1) * (1 if d == 0 else strides[d - 1]) for d in range(5))
        assert last == (1 << n) - 1
    assert sorted(covered) == list(range(n)), "every qubit in exactly one group"
    return groups


@pytest.mark.parametrize("variant", [0, 1, 3, 5])
@pytest.mark.parametrize("tma", [True, False])
def test_every_grouping_is_consistent(variant, tma):
    for n in range(8, 35):
        for tb in (0, 10, 11, 12, 13, 14):
            check_plan(n, tb, variant, tma)


def test_32_qubit_ring_plan():
    # the benchmark's plan: the low group on a 12-bit tile, the two strided
    # groups split so that they share the nine strided bits below bit 21 as
    # evenly as they can (4 and 5)
    g = check_plan(32, 13, 5, True)
    got = [(x.tile_bits, x.c, x.b, x.k, x.k1, x.b2) for x in g]
    assert got == [(12, 12, 12, 12, 12, 0), (13, 3, 12, 10, 4, 26), (13, 3, 16, 10, 10, 0)]
    low = sorted(sum(1 for q in rotated_bits(x, False) if q < SPREAD_BITS) for x in g[1:])
    assert low == [4, 5]


def test_refinements_need_the_ring():
    # without the tensor-map encoder, or off the ring variants, groups stay
    # contiguous and the low group keeps the main tile
    for tma, variant in ((False, 0), (True, 1), (True, 4)):
        g = check_plan(32, 13, variant, tma)
        assert g[0].tile_bits == 13 and all(x.k1 == x.k for x in g)


def test_no_extra_pass_for_the_smaller_low_tile():
    # the smaller low-group tile never costs a group: same count as a plain plan
    for n in range(15, 35):
        for tb in (11, 12, 13):
            assert len(check_plan(n, tb, 3, True)) == len(check_plan(n, tb, 3, False))


def test_24_qubit_ring_plan():
    # 24 qubits: both groups on 13-bit ring tiles, the 11 strided bits with 2
    # passenger bits (32-byte rows); one merged pass per Trotter step.  Forced
    # 14-bit tiles, another variant or no tensor-map encoder keep the 14 + 10
    # plan on the direct kernel; other sizes keep 3 or more passenger bits.
    g = check_plan(24, 0, 0, True)
    assert [(x.tile_bits, x.c, x.b, x.k) for x in g] == [(13, 13, 13, 13), (13, 2, 13, 11)]
    for tb, variant, tma in ((14, 0, True), (0, 1, True), (0, 0, False)):
        g = check_plan(24, tb, variant, tma)
        assert [(x.tile_bits, x.k) for x in g] == [(14, 14), (14, 10)]
    for n in (20, 22, 23, 25, 26):
        assert all(x.c >= 3 for x in check_plan(n, 0, 0, True)[1:])


def test_rejects_bad_arguments():
    for args in ((7, 0, 0, 0, True), (35, 0, 0, 0, True), (20, 5, 0, 0, True), (20, 0, 15, 0, True),
                 (20, 0, 0, 6, True)):
        with pytest.raises(z2.Z2Error):
            z2.z2_plan_geometry(*args)
