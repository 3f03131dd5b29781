"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads
and exports every entry point of include/z2lgt.h; the lattice builder is
bit-exact against the oracle's independent builder; argument errors come
back as status codes with messages."""

import os
import re
import subprocess

import numpy as np
import pytest

import paper_1910_08020_gb300 as z2
from oracle.lattice import Lattice as OLattice

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session", autouse=True)
def built():
    z2.build()
    z2.load()


def declared_entry_points():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(z2_\w+)\s*\(", txt, re.M))
    return names


def test_exports_every_declared_symbol():
    names = declared_entry_points()
    assert len(names) >= 18
    out = subprocess.run(["nm", "-D", "--defined-only", z2.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (z2_\w+)", out))
    missing = names - exported
    assert not missing, missing
    lib = z2.load()
    for n in names:
        assert getattr(lib, n) is not None


LATS = [(2, (2, 2)), (2, (3, 3)), (2, (4, 3)), (2, (4, 4)), (2, (5, 3)), (2, (3, 2)), (2, (2, 8)), (2, (8, 2)),
        (3, (2, 2, 2))]


@pytest.mark.parametrize("d,L", LATS)
def test_lattice_masks_bit_exact(d, L):
    lat = z2.Lattice(d, L)
    ref = OLattice(d, L)
    assert (lat.n_links, lat.n_plaq, lat.n_sites) == (ref.n_links, ref.n_plaq, ref.n_sites)
    assert np.array_equal(lat.masks(z2.Z2_MASK_PLAQ), ref.plaq_masks())
    assert np.array_equal(lat.masks(z2.Z2_MASK_STAR), ref.star_masks())
    assert np.array_equal(lat.masks(z2.Z2_MASK_W_MU), ref.w_masks())
    assert np.array_equal(lat.masks(z2.Z2_MASK_V_MU), ref.v_masks())
    w, _ = ref.wilson_2x2()
    assert int(lat.masks(z2.Z2_MASK_WILSON_2X2)[0]) == w
    assert [int(m) for m in lat.masks(z2.Z2_MASK_CONTOUR)] == [m for m, _ in ref.contours()]
    assert lat.state_bytes(z2.Z2_C64) == 8 << ref.n_links
    assert lat.state_bytes(z2.Z2_C128) == 16 << ref.n_links


@pytest.mark.parametrize("d,L", [(1, (4,)), (4, (2, 2)), (2, (1, 4)), (2, (6, 6)), (3, (3, 3, 3)), (3, (3, 2, 2)), (2, (8, 4))])
def test_lattice_errors(d, L):
    with pytest.raises(z2.Z2Error) as e:
        z2.Lattice(d, L)
    assert e.value.code in (-1, -2)
    assert len(str(e.value)) > 12


def test_mask_kind_error_and_version():
    lat = z2.Lattice(2, (3, 3))
    with pytest.raises(z2.Z2Error):
        lat.masks(99)
    assert "sm_103a" in z2.z2_version()


def _library_lattices():
    """Every lattice shape the library builds within its limits (2D L in
    2..17, 3D L in 2..3), found by asking it."""
    out = []
    for d, Ls in [(2, [(a, b) for a in range(2, 18) for b in range(2, 18)]),
                  (3, [(a, b, c) for a in (2, 3) for b in (2, 3) for c in (2, 3)])]:
        for L in Ls:
            try:
                lat = z2.Lattice(d, L)
            except Exception:
                continue
            out.append((d, L, lat.masks(z2.Z2_MASK_PLAQ), lat.n_links))
            lat.close()
    return out


def test_links_lie_in_few_plaquettes():
    """The pass kernels look up both phases of an amplitude pair (x, x ^ 1) in
    one table entry indexed by popcount(p) and popcount(p & c0), c0 the
    plaquette column of link 0, and reserve 8 entries per popcount(p) for the
    second index.  Every lattice the library builds keeps popcount(c0) at
    2 (d - 1), each link in exactly that many distinct plaquettes."""
    lats = _library_lattices()
    assert any(d == 3 for d, _, _, _ in lats) and len(lats) > 10
    for d, L, plaq, n_links in lats:
        counts = [sum(1 for m in plaq if (int(m) >> l) & 1) for l in range(n_links)]
        assert max(counts) < 8, (d, L)
        assert set(counts) == {2 * (d - 1)}, (d, L, set(counts))
