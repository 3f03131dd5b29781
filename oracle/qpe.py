"""Controlled time evolution for quantum phase estimation (Sec. 2.4, Eq. leap,
Fig. 5): TEST INFRASTRUCTURE ONLY, like the rest of `oracle/`.

For a fixed g, exp(-i H t) with H = Z + g X (Z = -sum_p U_p, X = -sum_l
sigma^x_l) is approximated by n Trotter steps of t/n, either
(exp(-i Z t/n) exp(-i g X t/n))^n, the X factor acting first, or the
symmetrised (exp(-i Z t/2n) exp(-i g X t/n) exp(-i Z t/2n))^n (Eq. leap).
Phase estimation needs U(t) = |0><0| (x) exp(-iHt) + |1><1| (x) exp(iHt): an
ancilla chooses the direction of time.  Here the ancilla is index bit N of a
state of 2^(N+1) amplitudes, so the half with the ancilla in |0> evolves for
+t and the other half for -t, each by the same Trotter formula.  For an
eigenstate |u> of H with energy E, (|0> + |1>)|u> / sqrt(2) becomes
(exp(-iEt)|0> + exp(iEt)|1>)|u> / sqrt(2), so <half 0|half 1> = exp(2iEt) / 2
up to the Trotter error, the quantity the paper's phase estimation reads out.

Layers as in the rest of the oracle: exp(-i Z tau) = D(tau) and
exp(-i g X tau) = R(g tau).
"""
import numpy as np

from . import FIRST_ORDER, SYMMETRIC, apply_D, apply_R
from .lattice import Lattice


def evolve_fixed_g(psi, lat: Lattice, g, t, n, decomp=SYMMETRIC):
    """exp(-i H t) psi for H = Z + g X by n Trotter steps (Eq. leap), in place
    on an N-link state; negative t runs time backwards."""
    if n < 1:
        raise ValueError("need n >= 1")
    masks = lat.plaq_masks()
    tau = t / n
    for _ in range(n):
        if decomp == FIRST_ORDER:
            apply_R(psi, g * tau)
            apply_D(psi, masks, tau)
        elif decomp == SYMMETRIC:
            apply_D(psi, masks, tau / 2)
            apply_R(psi, g * tau)
            apply_D(psi, masks, tau / 2)
        else:
            raise ValueError("bad decomposition")
    return psi


def controlled_evolution(psi, lat: Lattice, g, t, n, decomp=SYMMETRIC):
    """U(t) on a state of N + 1 qubits (ancilla = bit N), in place."""
    half = 1 << lat.n_links
    if len(psi) != 2 * half:
        raise ValueError("the state must hold 2^(N+1) amplitudes")
    evolve_fixed_g(psi[:half], lat, g, t, n, decomp)
    evolve_fixed_g(psi[half:], lat, g, -t, n, decomp)
    return psi


def ancilla_coherence(psi, n_links):
    """<half 0 | half 1> (complex): exp(2iEt)/2 for an eigenstate (see above)."""
    half = 1 << n_links
    return complex(np.vdot(psi[:half], psi[half:]))
