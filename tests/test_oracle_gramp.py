"""Pins of the oracle for the paper's own schedule, H(g) = Z + g X ramped from
g = 0 (oracle/gramp.py, Sec. 2.2-2.4), against facts that do not come from
the oracle itself:
- the start state by brute force over all link configurations, and the gauge
  and 't Hooft eigenvalues the paper states for it;
- at g = 0 the evolution is an exact global phase;
- substeps against dense matrix exponentials of Z and X built from their
  definitions (factor order, signs and the g_{k,m} sampling);
- the global order of the Trotter error with right-endpoint sampling;
- adiabatic convergence to the exact ground state of H(g_f).
"""
import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import FIRST_ORDER, SYMMETRIC, gramp
from oracle.ed import ground_state
from oracle.lattice import Lattice


def parities(n, masks):
    # parity of popcount(i & m) by folding the bits, independent of np.bitwise_count
    idx = np.arange(1 << n, dtype=np.uint64)
    out = []
    for m in masks:
        b = idx & np.uint64(m)
        for sh in (32, 16, 8, 4, 2, 1):
            b ^= b >> np.uint64(sh)
        out.append((b & np.uint64(1)).astype(np.int64))
    return np.array(out)


@pytest.mark.parametrize("d,L", [(2, (2, 2)), (2, (3, 3)), (3, (2, 2, 2))])
def test_start_state_is_the_projected_plus_state(d, L):
    lat = Lattice(d, L)
    n = lat.n_links
    psi = gramp.init_projected(lat)
    allowed = np.all(parities(n, lat.plaq_masks()) == 0, axis=0)  # U_p = +1 on every plaquette
    support = np.abs(psi) > 1e-12
    assert np.array_equal(support, allowed)
    amp = np.abs(psi[support])
    assert np.allclose(amp, amp[0], rtol=0, atol=1e-14) and abs(np.linalg.norm(psi) - 1) < 1e-13
    if d == 2:  # on a torus the plaquette constraints have exactly one dependency
        assert support.sum() == 2 ** (n - lat.n_plaq + 1)
    # ground state of Z (energy -N_p), Gauss law G_s = 1, 't Hooft V_mu = 1 (Sec. 2.4)
    assert abs(gramp.energy(lat, psi, 0.0) + lat.n_plaq) < 1e-12
    assert np.allclose(oracle.xsums(psi, lat.star_masks()), 1, atol=1e-12)
    assert np.allclose(oracle.xsums(psi, lat.v_masks()), 1, atol=1e-12)


@pytest.mark.parametrize("decomp", [FIRST_ORDER, SYMMETRIC])
def test_g_zero_is_a_global_phase(decomp):
    # with g_s = 0 every X factor is the identity and each Z factor multiplies
    # the all-U_p = +1 state by exp(i tau N_p): psi(T) = exp(i N_p N_s t_s) psi0
    lat = Lattice(2, (3, 3))
    psi0 = gramp.init_projected(lat)
    N_s, t_s = 3, 0.7
    psi = gramp.evolve_gramp(psi0.copy(), lat, 0.0, t_s, N_s, 5, decomp)
    assert np.max(np.abs(psi - np.exp(1j * lat.n_plaq * N_s * t_s) * psi0)) < 1e-12


def dense_Z_X(lat):
    n = lat.n_links
    par = parities(n, lat.plaq_masks())
    Z = np.diag(-np.sum(1 - 2 * par, axis=0).astype(np.float64))  # Z = sum_p Z_p, Z_p = -U_p
    X = np.zeros((1 << n, 1 << n))
    idx = np.arange(1 << n)
    for l in range(n):
        X[idx, idx ^ (1 << l)] -= 1.0                               # X = -sum_l sigma^x_l
    return Z, X


@pytest.mark.parametrize("decomp", [FIRST_ORDER, SYMMETRIC])
def test_substeps_match_dense_exponentials(decomp):
    lat = Lattice(2, (2, 2))
    Z, X = dense_Z_X(lat)
    g_s, t_s, N_s, n = 0.4, 0.9, 3, 4
    tau = t_s / n
    psi = gramp.init_projected(lat)
    want = psi.copy()
    for k in range(1, N_s + 1):
        for m in range(1, n + 1):
            g = (k - 1) * g_s + m * g_s / n
            ex = scipy.linalg.expm(-1j * g * X * tau)
            if decomp == FIRST_ORDER:
                want = scipy.linalg.expm(-1j * Z * tau) @ (ex @ want)
            else:
                half = scipy.linalg.expm(-1j * Z * tau / 2)
                want = half @ (ex @ (half @ want))
    got = gramp.evolve_gramp(psi, lat, g_s, t_s, N_s, n, decomp)
    assert np.max(np.abs(got - want)) < 1e-12
    # steps run in segments give the same state
    seg = gramp.init_projected(lat)
    gramp.evolve_gramp(seg, lat, g_s, t_s, N_s, n, decomp, 0, 1)
    gramp.evolve_gramp(seg, lat, g_s, t_s, N_s, n, decomp, 1, N_s)
    assert np.max(np.abs(seg - want)) < 1e-12


@pytest.mark.parametrize("decomp", [FIRST_ORDER, SYMMETRIC])
def test_right_endpoint_sampling_is_first_order(decomp):
    # g is held at the substep's right end (g_{k,m}), so even the symmetric split
    # converges at first order in t_s / n (the paper's error analysis leaves out
    # dH/dt): successive differences halve when n doubles
    lat = Lattice(2, (2, 2))
    g_s, t_s, N_s = 0.5, 2.0, 2
    states = []
    for n in (40, 80, 160, 320):
        states.append(gramp.evolve_gramp(gramp.init_projected(lat), lat, g_s, t_s, N_s, n, decomp))
    d = [np.linalg.norm(states[i] - states[i + 1]) for i in range(3)]
    for a, b in zip(d, d[1:]):
        assert 1.8 < a / b < 2.2, d


def test_slow_ramp_reaches_the_ground_state():
    # adiabatic theorem (Sec. 2.2): H_paper(g) = g * (-sum sigma^x - (1/g) sum U_p),
    # whose ground state in the V = + sector is that of the main path's H at
    # s*lambda = 1/g, found by Lanczos and pinned elsewhere by dense ED
    lat = Lattice(2, (2, 2))
    g_s, t_s, N_s, n = 0.05, 8.0, 12, 64          # g_f = 0.6, total time 96, tau = 0.125
    g_f = g_s * N_s
    psi = gramp.evolve_gramp(gramp.init_projected(lat), lat, g_s, t_s, N_s, n, SYMMETRIC)
    E0, phi0, r = ground_state(lat, 1.0 / g_f)
    assert r < 1e-10
    fid = abs(np.vdot(phi0, psi)) ** 2
    assert fid > 0.9995, fid
    assert abs(gramp.energy(lat, psi, g_f) - g_f * E0) < 2e-3 * lat.n_plaq


def test_rejects_bad_ramps():
    lat = Lattice(2, (2, 2))
    psi = gramp.init_projected(lat)
    for args in ((0.1, 1.0, 3, 0), (0.1, 1.0, 3, 4, SYMMETRIC, 2, 1), (0.1, 1.0, 3, 4, 7)):
        with pytest.raises(ValueError):
            gramp.evolve_gramp(psi.copy(), lat, *args)


@pytest.mark.parametrize("d,L", [(2, (2, 2)), (2, (3, 3)), (3, (2, 2, 2))])
def test_start_state_from_the_span_of_the_plaquette_masks(d, L):
    # a Hadamard layer maps prod_p (1 + U_p)/2 |+> to prod_p (1 + X_p)/2 |0>: the
    # uniform superposition over the GF(2) span of the plaquette masks (the
    # construction planned for the device), so the two must agree
    lat = Lattice(d, L)
    n = lat.n_links
    span = {0}
    for m in lat.plaq_masks():
        span |= {v ^ int(m) for v in span}
    r = len(span).bit_length() - 1
    assert len(span) == 1 << r
    if d == 2:
        assert r == lat.n_plaq - 1  # one dependency among the plaquettes of a torus
    phi = np.zeros(1 << n, dtype=np.complex128)
    phi[sorted(span)] = 2.0 ** (-r / 2)
    oracle.apply_hadamard_all(phi)
    assert np.max(np.abs(phi - gramp.init_projected(lat))) < 1e-12
