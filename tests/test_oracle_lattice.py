"""Pins for the oracle's lattice builder: the paper's printed counts and
plaquettes, and the algebra that gauge invariance rests on (checked by brute
force from the geometry, not from the builder's own formulas)."""

import os
from collections import Counter

import pytest

from oracle.lattice import Lattice

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_lattice.txt")


def _golden():
    counts, plaqs = [], []
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if f[0] == "counts":
            d = int(f[1])
            counts.append((d, tuple(map(int, f[2:2 + d])), int(f[2 + d]), int(f[3 + d])))
        else:
            plaqs.append(((int(f[1]), int(f[2])), set(map(int, f[3:7]))))
    return counts, plaqs


LATTICES = [(2, (2, 2)), (2, (3, 3)), (2, (4, 3)), (2, (4, 4)), (2, (5, 3)), (2, (3, 2)), (3, (2, 2, 2))]


def test_paper_counts():
    counts, _ = _golden()
    for d, L, nl, npq in counts:
        lat = Lattice(d, L)
        assert (lat.n_links, lat.n_plaq) == (nl, npq)


@pytest.mark.parametrize("d,L", LATTICES)
def test_counting_formulas(d, L):
    # N_l = d L^d and N_p = N_l (d-1)/2 (Sec. 2.1), generalised to L_x != L_y
    lat = Lattice(d, L)
    sites = 1
    for v in L:
        sites *= v
    assert lat.n_links == d * sites
    assert lat.n_plaq == lat.n_links * (d - 1) // 2


def test_paper_figure_plaquettes():
    _, plaqs = _golden()
    for (Lx, Ly), want in plaqs:
        lat = Lattice(2, (Lx, Ly))
        got = [set(lat.paper_link_number(l) for l in p) for p in lat.plaq_links]
        assert want in got


def _endpoints(lat, l):
    s, mu = divmod(l, lat.d)
    return s, lat.shift(s, mu, 1)


@pytest.mark.parametrize("d,L", LATTICES)
def test_plaquettes_are_closed_loops(d, L):
    lat = Lattice(d, L)
    per_link = Counter()
    for p in lat.plaq_links:
        assert len(set(p)) == 4
        deg = Counter()
        for l in p:
            a, b = _endpoints(lat, l)
            deg[a] += 1
            deg[b] += 1
            per_link[l] += 1
        assert all(v % 2 == 0 for v in deg.values())
    # every link borders 2(d-1) plaquettes
    assert set(per_link.values()) == {2 * (d - 1)}
    assert len(per_link) == lat.n_links


@pytest.mark.parametrize("d,L", LATTICES)
def test_stars_gauss_law_algebra(d, L):
    lat = Lattice(d, L)
    per_link = Counter()
    for s, st in enumerate(lat.star_links):
        assert len(set(st)) == 2 * d
        for l in st:
            assert s in _endpoints(lat, l)
            per_link[l] += 1
    assert set(per_link.values()) == {2}
    # G_s commutes with every U_p: even overlap (Sec. 2.1, G_i W_C G_i^-1 = W_C)
    for st in lat.star_links:
        for p in lat.plaq_links:
            assert len(set(st) & set(p)) % 2 == 0


@pytest.mark.parametrize("d,L", LATTICES)
def test_topological_loops(d, L):
    lat = Lattice(d, L)
    W = [set(l for l in range(lat.n_links) if (int(m) >> l) & 1) for m in lat.w_masks()]
    V = [set(l for l in range(lat.n_links) if (int(m) >> l) & 1) for m in lat.v_masks()]
    for mu in range(d):
        # W_mu is a closed loop winding once around direction mu
        deg = Counter()
        for l in W[mu]:
            a, b = _endpoints(lat, l)
            deg[a] += 1
            deg[b] += 1
        assert all(v == 2 for v in deg.values())
        assert len(W[mu]) == L[mu]
        # V_mu commutes with H (every plaquette) and every star trivially
        for p in lat.plaq_links:
            assert len(V[mu] & set(p)) % 2 == 0
        for st in lat.star_links:
            assert len(W[mu] & set(st)) % 2 == 0
        for nu in range(d):
            # W anticommutes with exactly one surface operator (Sec. 2.1)
            assert (len(W[mu] & V[nu]) % 2 == 1) == (mu == nu)


def _perimeter(m):
    return bin(int(m)).count("1")


def test_contours_perimeter_ratio():
    # Sec. 3.1: contours c1, c2, c3 with perimeters in ratio 1 : 1.5 : 2
    for d, L in [(2, (3, 3)), (2, (4, 4)), (3, (2, 2, 2))]:
        lat = Lattice(d, L)
        per = [_perimeter(m) for m, deg in lat.contours()]
        assert per == [4, 6, 8]
        assert not any(deg for _, deg in lat.contours())
    w, deg = Lattice(2, (3, 3)).wilson_2x2()
    assert _perimeter(w) == 8 and not deg
    assert Lattice(2, (2, 2)).wilson_2x2() == (0, True)
    assert Lattice(3, (2, 2, 2)).wilson_2x2()[1]


def test_rejects_bad_lattices():
    for d, L in [(1, (3,)), (2, (1, 3)), (2, (3,)), (4, (2, 2, 2, 2))]:
        with pytest.raises(ValueError):
            Lattice(d, L)
