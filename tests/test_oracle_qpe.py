"""Pins of the oracle for the controlled evolution of phase estimation
(oracle/qpe.py, Sec. 2.4, Eq. leap), against facts that do not come from the
oracle itself:
- the Trotter formulas against products of dense matrix exponentials of Z and
  X built from their definitions (factor order and signs);
- convergence to the exact exp(-iHt) (dense expm) at first and second order;
- the paper's own error estimates for the two formulas, 2 g N_p t^2 / n and
  ((d-1) g + 4 g^2) / 3 N_p t^3 / n^2, as bounds on the state error;
- the ancilla choosing the direction of time, against the exact block
  diagonal exp(-iHt) (+) exp(iHt);
- the phase read out from an eigenstate of a dense diagonalisation;
- exact time reversal of the symmetrised formula.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import FIRST_ORDER, SYMMETRIC, qpe
from oracle.lattice import Lattice
from test_oracle_gramp import dense_Z_X


def rand_state(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return v / np.linalg.norm(v)


def paper_bound(decomp, lat, g, t, n):
    # the two estimates printed after Eq. (leap)
    if decomp == FIRST_ORDER:
        return 2 * g * lat.n_plaq * t ** 2 / n
    return ((lat.d - 1) * g + 4 * g * g) / 3 * lat.n_plaq * t ** 3 / n ** 2


@pytest.mark.parametrize("decomp", [FIRST_ORDER, SYMMETRIC])
def test_trotter_formula_matches_dense_factors(decomp):
    lat = Lattice(2, (2, 2))
    Z, X = dense_Z_X(lat)
    g, t, n = 0.8, 1.3, 5
    tau = t / n
    v = rand_state(lat.n_links, 1)
    want = v.copy()
    ez, ex, ez2 = (scipy.linalg.expm(-1j * Z * tau), scipy.linalg.expm(-1j * g * X * tau),
                   scipy.linalg.expm(-1j * Z * tau / 2))
    for _ in range(n):
        want = ez @ (ex @ want) if decomp == FIRST_ORDER else ez2 @ (ex @ (ez2 @ want))
    got = qpe.evolve_fixed_g(v.copy(), lat, g, t, n, decomp)
    assert np.max(np.abs(got - want)) < 1e-12


@pytest.mark.parametrize("decomp,order", [(FIRST_ORDER, 1), (SYMMETRIC, 2)])
def test_convergence_order_against_exact_evolution(decomp, order):
    lat = Lattice(2, (2, 2))
    Z, X = dense_Z_X(lat)
    g, t = 1.1, 0.9
    U = scipy.linalg.expm(-1j * (Z + g * X) * t)
    v = rand_state(lat.n_links, 2)
    err = [np.linalg.norm(qpe.evolve_fixed_g(v.copy(), lat, g, t, n, decomp) - U @ v) for n in (10, 40, 160)]
    for a, b in zip(err, err[1:]):
        assert 0.85 * 4 ** order < a / b < 1.15 * 4 ** order, err


@pytest.mark.parametrize("decomp", [FIRST_ORDER, SYMMETRIC])
@pytest.mark.parametrize("g,t", [(0.5, 0.5), (0.5, 2.0), (1.5, 0.5), (1.5, 2.0)])
def test_paper_error_estimates_bound_the_state_error(decomp, g, t):
    lat = Lattice(2, (2, 2))
    Z, X = dense_Z_X(lat)
    U = scipy.linalg.expm(-1j * (Z + g * X) * t)
    for n in (10, 40):
        for seed in range(4):
            v = rand_state(lat.n_links, 10 + seed)
            e = np.linalg.norm(qpe.evolve_fixed_g(v.copy(), lat, g, t, n, decomp) - U @ v)
            assert e <= paper_bound(decomp, lat, g, t, n)


@pytest.mark.parametrize("decomp", [FIRST_ORDER, SYMMETRIC])
def test_ancilla_chooses_the_direction_of_time(decomp):
    lat = Lattice(2, (2, 2))
    Z, X = dense_Z_X(lat)
    N = lat.n_links
    g, t, n = 0.7, 0.6, 60
    H = Z + g * X
    exact = scipy.linalg.block_diag(scipy.linalg.expm(-1j * H * t), scipy.linalg.expm(1j * H * t))
    v = rand_state(N + 1, 3)
    got = qpe.controlled_evolution(v.copy(), lat, g, t, n, decomp)
    assert np.linalg.norm(got - exact @ v) <= paper_bound(decomp, lat, g, t, n)
    # and the halves are exactly the forward and backward Trotter evolutions
    lo = qpe.evolve_fixed_g(v[: 1 << N].copy(), lat, g, t, n, decomp)
    hi = qpe.evolve_fixed_g(v[1 << N:].copy(), lat, g, -t, n, decomp)
    assert np.array_equal(got, np.concatenate([lo, hi]))


@pytest.mark.parametrize("decomp", [FIRST_ORDER, SYMMETRIC])
def test_phase_of_an_eigenstate(decomp):
    # (|0> + |1>)|u>/sqrt(2) -> (e^{-iEt}|0> + e^{iEt}|1>)|u>/sqrt(2): the
    # ancilla coherence <half 0|half 1> = e^{2iEt}/2, for E from eigh
    lat = Lattice(2, (2, 2))
    Z, X = dense_Z_X(lat)
    N = lat.n_links
    g, t, n = 0.9, 0.7, 200
    w, V = np.linalg.eigh(Z + g * X)
    for k in (0, 5, 37):
        u = V[:, k].astype(np.complex128)
        psi = np.concatenate([u, u]) / np.sqrt(2)
        qpe.controlled_evolution(psi, lat, g, t, n, decomp)
        c = qpe.ancilla_coherence(psi, N)
        assert abs(c - np.exp(2j * w[k] * t) / 2) <= paper_bound(decomp, lat, g, t, n)


def test_symmetric_formula_is_time_reversible():
    lat = Lattice(2, (3, 3))
    v = rand_state(lat.n_links, 4)
    w = qpe.evolve_fixed_g(v.copy(), lat, 1.2, 0.8, 7, SYMMETRIC)
    qpe.evolve_fixed_g(w, lat, 1.2, -0.8, 7, SYMMETRIC)
    assert np.max(np.abs(w - v)) < 1e-12


def test_rejects_bad_arguments():
    lat = Lattice(2, (2, 2))
    with pytest.raises(ValueError):
        qpe.evolve_fixed_g(rand_state(8, 0), lat, 1.0, 1.0, 0)
    with pytest.raises(ValueError):
        qpe.evolve_fixed_g(rand_state(8, 0), lat, 1.0, 1.0, 3, 7)
    with pytest.raises(ValueError):
        qpe.controlled_evolution(rand_state(8, 0), lat, 1.0, 1.0, 3)
