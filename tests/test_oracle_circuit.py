"""The fused plaquette layer is the paper's gate-level circuit (Sec. 2.3,
Eq. ara, Fig. 3): simulating the four-CNOT / R_z / four-CNOT sequence with one
ancilla for every plaquette gives exactly the diagonal layer D(tau) that the
kernels apply as one table lookup, and leaves the ancilla in |0>."""
import numpy as np
import pytest

import oracle
from oracle.circuit import apply_plaquettes_with_ancilla
from oracle.lattice import Lattice


@pytest.mark.parametrize("d,L", [(2, (2, 2)), (2, (3, 3))])
@pytest.mark.parametrize("tau", [0.13, -0.7, 2.4])
def test_ancilla_circuit_equals_the_fused_diagonal(d, L, tau):
    lat = Lattice(d, L)
    n = lat.n_links
    rng = np.random.default_rng(11)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi /= np.linalg.norm(psi)
    got, leak = apply_plaquettes_with_ancilla(psi, lat.plaq_masks(), tau)
    want = oracle.apply_D(psi.copy(), lat.plaq_masks(), tau)  # exp(-i Z tau) = D(tau), Z = -sum U_p
    assert leak < 1e-14
    assert np.max(np.abs(got - want)) < 1e-13
