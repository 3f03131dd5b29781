"""Pins for the oracle's exact diagonalisation, Lanczos solver, Magnus
reference integrator and the 2+1D duality simulator: textbook spectra,
library routines (numpy.linalg.eigh, scipy.linalg.expm, scipy ODE solver),
the paper's gap statements, and the exact gauge/Ising duality."""

import math

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

import oracle
from oracle import ed
from oracle.dual import DualIsing
from oracle.lattice import Lattice


def sector_projector(lat):
    """Projector on G_s = 1 for all s and V_mu = +1, as dense products of
    (1 + O)/2 with O = prod sigma^x (a bit-flip permutation matrix)."""
    dim = 1 << lat.n_links
    rows = np.arange(dim)
    P = np.eye(dim)
    for m in list(lat.star_masks()) + list(lat.v_masks()):
        O = np.zeros((dim, dim))
        O[rows ^ int(m), rows] = 1.0
        P = P @ (0.5 * (np.eye(dim) + O))
    return P


def test_dense_h_lambda_zero_spectrum():
    # H = -sum_l sigma^x_l: eigenvalues -N + 2w with multiplicity C(N, w)
    lat = Lattice(2, (2, 2))
    ev = np.linalg.eigvalsh(ed.hamiltonian_dense(lat, 0.0))
    n = lat.n_links
    want = sorted(-n + 2 * w for w in range(n + 1) for _ in range(math.comb(n, w)))
    assert np.allclose(ev, want, atol=1e-12)


def test_dense_h_matches_oracle_matvec():
    lat = Lattice(2, (3, 2))
    rng = np.random.default_rng(5)
    x = rng.normal(size=1 << lat.n_links) + 1j * rng.normal(size=1 << lat.n_links)
    H = ed.hamiltonian_dense(lat, 1.3)
    assert np.allclose(H @ x, oracle.hamiltonian_apply(lat, x, 1.3), atol=1e-12)
    assert np.allclose(ed.SparseH(lat, 1.3)(x.real), H @ x.real, atol=1e-12)


@pytest.mark.parametrize("slam", [0.0, 0.7, 3.0, 10.0])
def test_lanczos_vs_eigh_in_sector(slam):
    lat = Lattice(2, (2, 2))
    H = ed.hamiltonian_dense(lat, slam)
    P = sector_projector(lat)
    # the sector ground state: lowest eigenvalue of P H P on range(P)
    U, s, _ = np.linalg.svd(P)
    B = U[:, s > 0.5]
    assert B.shape[1] == 1 << (lat.n_plaq - 1)  # sector dimension 2^{N_p - 1}
    evs = np.linalg.eigvalsh(B.T @ H @ B)
    E, phi, r = ed.ground_state(lat, slam)
    assert r < 1e-10
    assert abs(E - evs[0]) < 1e-10
    if slam == 0.0:
        # Sec. 2.6: in the strong-coupling limit the gauge-invariant gap is 8
        # (flipping sigma^x on the four links of one plaquette)
        assert abs(evs[0] + lat.n_links) < 1e-12
        assert abs(evs[1] - evs[0] - 8) < 1e-12
    # the sector ground state is the global ground state for s*lambda > 0 or
    # degenerate with it (Sec. 2.1: V = + holds the ground state)
    assert evs[0] <= np.linalg.eigvalsh(H)[0] + 1e-10


def test_weak_coupling_gap():
    # Sec. 2.6: deep in the deconfined phase the lowest excitation is a pair
    # of visons costing 4 in paper units; with H = -X - lambda*sum U_p that is
    # 4*lambda to leading order (the V = + sector, 3x3 through the dual)
    lat = Lattice(2, (3, 3))
    du = DualIsing(lat)
    lam = 2000.0
    H = np.zeros((1 << du.n, 1 << du.n))
    for i in range(1 << du.n):
        e = np.zeros(1 << du.n)
        e[i] = 1
        H[:, i] = du.hamiltonian_apply(e, lam)
    # restrict to the even sector
    idx = np.arange(1 << du.n)
    comp = idx ^ ((1 << du.n) - 1)
    evenB = np.zeros((1 << du.n, 1 << (du.n - 1)))
    k = 0
    for i in range(1 << du.n):
        if i < comp[i]:
            evenB[i, k] = evenB[comp[i], k] = 1 / np.sqrt(2)
            k += 1
    ev = np.linalg.eigvalsh(evenB.T @ H @ evenB)
    gap = ev[1] - ev[0]
    assert abs(gap / lam - 4) < 0.01


def test_magnus_constant_h_is_exact():
    lat = Lattice(2, (2, 2))
    psi = ed.magnus4_evolution(lat, 0.0, 1.3, 3)
    H = ed.hamiltonian_dense(lat, 0.0)
    want = scipy.linalg.expm(-1j * 1.3 * H) @ np.full(256, 1 / 16, dtype=complex)
    assert np.max(np.abs(psi - want)) < 1e-13


def test_magnus_vs_library_ode():
    lat = Lattice(2, (2, 2))
    lam, T = 2.0, 1.0
    H0 = ed.hamiltonian_dense(lat, 0.0)
    P = -ed.plaquette_diagonal(lat)

    def f(t, y):
        psi = y[:256] + 1j * y[256:]
        d = -1j * (H0 @ psi + lam * (t / T) * P * psi)
        return np.concatenate([d.real, d.imag])

    y0 = np.concatenate([np.full(256, 1 / 16), np.zeros(256)])
    sol = scipy.integrate.solve_ivp(f, (0, T), y0, method="DOP853", rtol=1e-12, atol=1e-13)
    ref = sol.y[:256, -1] + 1j * sol.y[256:, -1]
    psi = ed.magnus4_evolution(lat, lam, T, 200)
    assert np.max(np.abs(psi - ref)) < 1e-9


def test_trotter_order_against_magnus():
    # the schemes approximate the time-ordered evolution: errors fall as dt
    # (first order) and dt^2 (symmetric, trapezoid halves); the paper's literal
    # right-end sampling of both symmetric halves ignores dH/dt and is only
    # O(dt) for a ramped H
    lat = Lattice(2, (2, 2))
    lam, T = 3.0, 2.0
    exact = ed.magnus4_evolution(lat, lam, T, 100)
    Ms = (200, 400, 800)
    ratio = {}
    for dec, samp in ((0, 0), (1, 0), (1, 1)):
        e = [np.linalg.norm(oracle.run(lat, lam, T, M, dec, samp) - exact) for M in Ms]
        ratio[dec, samp] = e[1] / e[2]
    assert 1.9 < ratio[0, 0] < 2.1
    assert 3.9 < ratio[1, 0] < 4.1
    assert 1.9 < ratio[1, 1] < 2.1


# -- duality -------------------------------------------------------------------
@pytest.mark.parametrize("L,lam,decomp,M", [((3, 3), 1.0, 1, 60), ((3, 2), 3.0, 0, 50), ((2, 2), 2.0, 1, 30)])
def test_dual_dynamics_match_direct(L, lam, decomp, M):
    lat = Lattice(2, L)
    T = 3.0
    psi = oracle.run(lat, lam, T, M, decomp)
    ob = oracle.observables(lat, psi, lam)
    du = DualIsing(lat)
    ob2 = du.observables(du.run(lam, T, M, decomp), lam)
    assert abs(ob["energy"] - ob2["energy"]) < 1e-11
    assert np.allclose(ob["plaq"], ob2["plaq"], atol=1e-12)
    assert np.allclose(ob["sigmax"], ob2["sigmax"], atol=1e-12)
    if not np.isnan(ob["wilson_2x2"]):
        assert abs(ob["wilson_2x2"] - ob2["wilson_2x2"]) < 1e-12


def test_dual_ground_state_and_fidelity():
    lat = Lattice(2, (3, 3))
    lam, T, M = 1.0, 4.0, 80
    E, phi, r = ed.ground_state(lat, lam)
    du = DualIsing(lat)
    E2, phi2, r2 = du.ground_state(lam)
    assert r < 1e-9 and r2 < 1e-10
    assert abs(E - E2) < 1e-9
    F = abs(oracle.overlap(phi, oracle.run(lat, lam, T, M, 1))) ** 2
    F2 = abs(np.vdot(phi2, du.run(lam, T, M, 1))) ** 2
    assert abs(F - F2) < 1e-9


def test_dual_sector_dimension():
    # 3x3: 2^{18 - 8 - 2} = 256 = 2^9 / 2 (Gauss law removes sites-1 bits,
    # the 't Hooft loops two more; the dual keeps the Z2-even half)
    lat = Lattice(2, (3, 3))
    assert lat.n_links - (lat.n_sites - 1) - 2 == lat.n_plaq - 1
