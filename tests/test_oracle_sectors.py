"""Pins of the topological-sector part of the paper's own schedule
(oracle/gramp.py: sector_start, sector_ground_state; Sec. 2.1, 2.4 and 4.3):
- the 't Hooft eigenvalues of each sector start follow from the masks alone
  (W_mu anticommutes with V_nu iff their link sets share an odd number of links);
- sector energies against dense exact diagonalisation with projectors built
  from the gauge and 't Hooft operators (2x2 lattice, independent of Lanczos);
- E(-1, 1) = E(1, -1) on L x L tori (the x <-> y symmetry, Sec. 4.3);
- the small-g splitting E_21 grows as g^L: the lowest perturbative process
  between sectors flips the L links crossed by a non-contractible dual loop;
- an adiabatic ramp started in a sector keeps its 't Hooft eigenvalues and ends
  in that sector's lowest state.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import SYMMETRIC, gramp
from oracle.lattice import Lattice


def popc(v):
    return bin(int(v)).count("1")


@pytest.mark.parametrize("d,L", [(2, (2, 2)), (2, (3, 3)), (3, (2, 2, 2))])
def test_sector_start_flips_the_crossed_thooft_operators(d, L):
    lat = Lattice(d, L)
    w, v = lat.w_masks(), lat.v_masks()
    start = gramp.init_projected(lat)
    for r in range(d + 1):
        for flips in itertools.combinations(range(d), r):
            psi = gramp.sector_start(lat, flips, start)
            want = [np.prod([(-1) ** popc(int(w[mu]) & int(v[nu])) for mu in flips]) for nu in range(d)]
            assert np.allclose(oracle.xsums(psi, v).real, want, atol=1e-12), (flips, want)
            assert np.allclose(oracle.xsums(psi, lat.star_masks()), 1, atol=1e-12)
            assert abs(gramp.energy(lat, psi, 0.0) + lat.n_plaq) < 1e-12


def perm(n, m):
    """prod_{l in m} sigma^x_l as a dense permutation matrix."""
    P = np.zeros((1 << n, 1 << n))
    i = np.arange(1 << n)
    P[i ^ int(m), i] = 1.0
    return P


def dense_sector_energies(lat, g):
    n = lat.n_links
    i = np.arange(1 << n)
    U = np.zeros(1 << n)
    for m in lat.plaq_masks():
        U += np.array([1 - 2 * (popc(k & int(m)) & 1) for k in i])
    H = np.diag(-U)                               # Z = -sum_p U_p
    for l in range(n):
        H -= g * perm(n, 1 << l)                  # + g X, X = -sum_l sigma^x_l
    G = np.eye(1 << n)
    for s in lat.star_masks():
        G = G @ (np.eye(1 << n) + perm(n, s)) / 2
    out = {}
    for signs in itertools.product((1, -1), repeat=lat.d):
        P = G.copy()
        for mu, sgn in enumerate(signs):
            P = P @ (np.eye(1 << n) + sgn * perm(n, lat.v_masks()[mu])) / 2
        evals, evecs = np.linalg.eigh(P)
        Q = evecs[:, evals > 0.5]
        out[signs] = np.linalg.eigvalsh(Q.T @ H @ Q)[0]
    return out


@pytest.mark.parametrize("g", [0.2, 0.5, 1.5])
def test_sector_energies_match_dense_diagonalisation(g):
    lat = Lattice(2, (2, 2))
    dense = dense_sector_energies(lat, g)
    w, v = lat.w_masks(), lat.v_masks()
    for r in range(3):
        for flips in itertools.combinations(range(2), r):
            signs = tuple(int(np.prod([(-1) ** popc(int(w[mu]) & int(v[nu])) for mu in flips])) for nu in range(2))
            E, phi, res = gramp.sector_ground_state(lat, g, flips)
            assert res < 1e-10
            assert abs(E - dense[signs]) < 1e-9, (flips, E, dense[signs])


def test_equal_splittings_by_symmetry():
    lat = Lattice(2, (3, 3))
    g = 0.25
    E1 = gramp.sector_ground_state(lat, g, [])[0]
    E2 = gramp.sector_ground_state(lat, g, [0])[0]
    E3 = gramp.sector_ground_state(lat, g, [1])[0]
    E4 = gramp.sector_ground_state(lat, g, [0, 1])[0]
    assert abs(E2 - E3) < 1e-9 and E1 < E2 < E4


@pytest.mark.parametrize("L,gs", [(2, (0.01, 0.02, 0.04)), (3, (0.02, 0.04))])
def test_small_g_splitting_goes_as_g_to_the_L(L, gs):
    lat = Lattice(2, (L, L))
    gs = np.array(gs)
    split = [gramp.sector_ground_state(lat, g, [0])[0] - gramp.sector_ground_state(lat, g, [])[0] for g in gs]
    slopes = np.diff(np.log(split)) / np.diff(np.log(gs))
    assert np.all(np.abs(slopes - L) < 0.1), slopes


def test_ramp_stays_in_its_sector():
    lat = Lattice(2, (2, 2))
    g_s, t_s, N_s, n = 0.05, 8.0, 12, 64
    g_f = g_s * N_s
    psi = gramp.evolve_gramp(gramp.sector_start(lat, [0]), lat, g_s, t_s, N_s, n, SYMMETRIC)
    assert np.allclose(oracle.xsums(psi, lat.v_masks()).real, [-1, 1], atol=1e-10)
    E, phi, r = gramp.sector_ground_state(lat, g_f, [0])
    assert abs(np.vdot(phi, psi)) ** 2 > 0.9995
