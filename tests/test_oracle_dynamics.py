"""Pins for the oracle's state-vector dynamics and observables: closed forms,
brute force, invariants of the gauge theory, convergence order, and the
schedule sums printed in the paper."""

import math
import os

import numpy as np
import pytest

import oracle
from oracle import schedule
from oracle.lattice import Lattice

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_error_estimates.txt")


def basis(n, i):
    v = np.zeros(1 << n, dtype=np.complex128)
    v[i] = 1.0
    return v


def odd_plaquettes_bruteforce(lat, i):
    """Number of plaquettes whose four link bits hold an odd number of ones,
    read from the link lists (no masks)."""
    return sum(sum((i >> l) & 1 for l in p) % 2 for p in lat.plaq_links)


def test_init_plus():
    psi = oracle.init_plus(10)
    assert np.allclose(psi, 2 ** -5)
    assert abs(np.vdot(psi, psi) - 1) < 1e-15


@pytest.mark.parametrize("w_i", [0, 1, 0b1011, 0b111111])
def test_R_on_basis_state_closed_form(w_i):
    # R(dt)|i> = prod_l (cos dt |i_l> + i sin dt |1-i_l>): amplitude on |j> is
    # cos^{n-w} (i sin)^w with w = popcount(i ^ j)
    n, dt = 6, 0.37
    psi = oracle.apply_R(basis(n, w_i), dt)
    for j in range(1 << n):
        w = bin(w_i ^ j).count("1")
        want = math.cos(dt) ** (n - w) * (1j * math.sin(dt)) ** w
        assert abs(psi[j] - want) < 1e-14


@pytest.mark.parametrize("d,L", [(2, (3, 3)), (2, (2, 2)), (3, (2, 2, 2))])
def test_D_on_basis_states_bruteforce(d, L):
    lat = Lattice(d, L)
    rng = np.random.default_rng(7)
    theta = 0.213
    for i in rng.integers(0, 1 << lat.n_links, size=40 if lat.n_links <= 18 else 4):
        psi = oracle.apply_D(basis(lat.n_links, int(i)), lat.plaq_masks(), theta)
        k = odd_plaquettes_bruteforce(lat, int(i))
        want = np.exp(1j * theta * (lat.n_plaq - 2 * k))
        assert abs(psi[int(i)] - want) < 1e-14
        assert np.count_nonzero(psi) == 1


def test_zdos_bruteforce_counts():
    lat = Lattice(2, (2, 2))
    n = lat.n_links
    rng = np.random.default_rng(3)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi /= np.linalg.norm(psi)
    want = np.zeros(lat.n_plaq + 1)
    for i in range(1 << n):
        want[odd_plaquettes_bruteforce(lat, i)] += abs(psi[i]) ** 2
    assert np.allclose(oracle.zdos(psi, lat.plaq_masks()), want, atol=1e-14)


@pytest.mark.parametrize("decomp", [0, 1])
def test_lambda_zero_closed_form(decomp):
    # lambda = 0: H = -sum sigma^x and |+>^N is its eigenstate, so
    # psi(T) = exp(i N T)|+>^N exactly for both decompositions (D(0) = 1)
    lat = Lattice(2, (3, 3))
    T, M = 1.7, 30
    psi = oracle.run(lat, 0.0, T, M, decomp)
    want = np.exp(1j * lat.n_links * T) * 2 ** (-lat.n_links / 2)
    assert np.max(np.abs(psi - want)) < 1e-13


def test_unitarity_random_state():
    lat = Lattice(2, (3, 2))
    n = lat.n_links
    rng = np.random.default_rng(11)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi /= np.linalg.norm(psi)
    ref = psi.copy()
    oracle.evolve(psi, lat.plaq_masks(), 2.5, 3.0, 40, decomp=1)
    assert abs(np.vdot(psi, psi) - 1) < 1e-13
    # inner products are preserved too: evolve a second state
    phi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    phi /= np.linalg.norm(phi)
    ov0 = np.vdot(phi, ref)
    oracle.evolve(phi, lat.plaq_masks(), 2.5, 3.0, 40, decomp=1)
    assert abs(np.vdot(phi, psi) - ov0) < 1e-13


def test_xsums_equal_hadamard_then_zsums():
    # <prod sigma^x> computed from the permutation sum equals the sigma^z sum
    # after a Hadamard on every qubit (H sigma^z H = sigma^x, Sec. 2.4)
    lat = Lattice(2, (2, 2))
    psi = oracle.run(lat, 2.0, 2.0, 20, 1)
    masks = np.concatenate([lat.star_masks(), lat.v_masks(), [1 << l for l in range(lat.n_links)]])
    masks = masks.astype(np.uint64)
    direct = oracle.xsums(psi, masks)
    viaH = oracle.zsums(oracle.apply_hadamard_all(psi.copy()), masks)
    assert np.allclose(direct.real, viaH, atol=1e-13)
    assert np.allclose(direct.imag, 0, atol=1e-13)


_RUNS = {}


def _run_cached(d, L, lam, T, M):
    key = (d, L, lam, T, M)
    if key not in _RUNS:
        _RUNS[key] = oracle.run(Lattice(d, L), lam, T, M, 1)
    return _RUNS[key]


@pytest.mark.parametrize("d,L,lam", [(2, (3, 3), 1.0), (3, (2, 2, 2), 1.5)])
def test_gauge_invariants_after_run(d, L, lam):
    # Sec. 2.3: every substep is gauge invariant, so G_s = 1 stays exact; the
    # run stays in the V = + sector where <W_mu> = 0 (W anticommutes with V),
    # <sigma^z_l> = 0 (Sec. 3.5), the norm is 1 and translation symmetry makes
    # all <U_p> of one orientation equal.
    lat = Lattice(d, L)
    M = 6 if d == 3 else 20
    psi = _run_cached(d, L, lam, 2.0, M)
    ob = oracle.observables(lat, psi, lam)
    assert abs(ob["norm"] - 1) < 1e-11
    assert np.allclose(ob["star"], 1, atol=1e-11)
    assert np.allclose(ob["vmu"], 1, atol=1e-11)
    assert np.allclose(ob["wmu"], 0, atol=1e-11)
    assert np.allclose(ob["sigmaz"], 0, atol=1e-11)
    assert np.ptp(ob["plaq"]) < 1e-11
    assert np.ptp(ob["sigmax"]) < 1e-11
    assert abs(ob["zdos"].sum() - 1) < 1e-11


def test_zdos_support_3d():
    # Sec. 3.3: on the 2x2x2 lattice the Z eigenvalue z = -sum U_p never takes
    # the values +-20 (k = 2 or 22 odd plaquettes): that mass must vanish
    lat = Lattice(3, (2, 2, 2))
    psi = _run_cached(3, (2, 2, 2), 1.5, 2.0, 6)
    dos = oracle.zdos(psi, lat.plaq_masks())
    assert dos[2] < 1e-28 and dos[22] < 1e-28
    # and since every link borders 4 plaquettes, k is always even
    assert np.all(dos[1::2] < 1e-28)


def test_zdos_support_2d():
    # Sec. 3.3 (2D): z takes the values -9 + 4n on the 3x3 lattice, i.e. the
    # number of odd plaquettes is even (each link borders two plaquettes)
    lat = Lattice(2, (3, 3))
    psi = _run_cached(2, (3, 3), 1.0, 2.0, 20)
    dos = oracle.zdos(psi, lat.plaq_masks())
    assert np.all(dos[1::2] < 1e-28)


def test_segmented_equals_whole():
    lat = Lattice(2, (3, 2))
    a = oracle.run(lat, 3.0, 4.0, 30, 1)
    b = oracle.init_plus(lat.n_links)
    for j0, j1 in [(0, 7), (7, 8), (8, 30)]:
        oracle.evolve(b, lat.plaq_masks(), 3.0, 4.0, 30, 1, j0=j0, j1=j1)
    assert np.array_equal(a, b)


def _order(lat, lam, T, decomp, sampling, Ms):
    states = [oracle.run(lat, lam, T, M, decomp, sampling) for M in Ms]
    diffs = [np.linalg.norm(states[k] - states[k + 1]) for k in range(len(Ms) - 1)]
    return [diffs[k] / diffs[k + 1] for k in range(len(diffs) - 1)]


def test_convergence_order():
    # Eq. (asymtotal) vs Eq. (total): first order converges as O(dt), the
    # symmetric (trapezoid) split as O(dt^2).
    lat = Lattice(2, (3, 2))
    Ms = [50, 100, 200, 400]
    r1 = _order(lat, 2.0, 3.0, 0, 0, Ms)
    r2 = _order(lat, 2.0, 3.0, 1, 0, Ms)
    assert 1.8 < r1[-1] < 2.2
    assert 3.7 < r2[-1] < 4.3


def test_schedule_sums_closed_form():
    # Sec. 2.2: the closed-form sums of g_{k,m} and g_{k,m}^2 pin the
    # right-end sampling of each substep
    for N_s, n, g_s in [(7, 3, 0.25), (20, 11, 0.001), (1, 5, 1.0)]:
        g = schedule.g_values(N_s, n, g_s)
        assert abs(sum(g) - schedule.sum_g_closed(N_s, n, g_s)) < 1e-12 * max(1, sum(g))
        s2 = sum(x * x for x in g)
        assert abs(s2 - schedule.sum_g2_closed(N_s, n, g_s)) < 1e-12 * max(1, s2)


def test_paper_error_estimates():
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        kind, d, N_p, t_s, n, printed, tol = line.split()
        args = (2000, int(N_p), 0.001, float(t_s), int(n))
        val = schedule.delta_sym_total(*args) if kind == "sym" else schedule.delta_asym_total(*args)
        assert abs(val - float(printed)) <= float(tol) * float(printed), (kind, d, val)


def test_xdos_support():
    # Sec. 3.3: gauge invariance forces the links flipped in the sigma^x basis
    # to form closed loops of perimeter 4 + 2n, so w (the number of sigma^x = -1
    # links) is 0 or 4, 6, 8, ... on both lattices; in 3D also w != N - 2
    # (x = +-20 absent, self-duality).  The all-flipped state has V = -1 on the
    # 3x3 lattice (odd loop length), so inside the V = + sector w = 18 is absent.
    for d, L, lam, M in [(2, (3, 3), 1.0, 20), (3, (2, 2, 2), 1.5, 6)]:
        lat = Lattice(d, L)
        psi = _run_cached(d, L, lam, 2.0, M)
        dos = oracle.xdos(psi)
        n = lat.n_links
        allowed = {0} | set(range(4, n + 1, 2))
        if d == 3:
            allowed -= {n - 2}
        else:
            allowed -= {n}
        for w in range(n + 1):
            if w not in allowed:
                assert dos[w] < 1e-26, (d, w, dos[w])
        assert abs(dos.sum() - 1) < 1e-12
